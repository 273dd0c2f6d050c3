// Particle order by mesh cell: a stable least-significant-digit radix sort
// of the particles on the cell of their CIC base node, then one gather of
// the float4 records into the new order.  It changes no result of a step
// (every per-particle update is independent of the order and the deposit
// sums integers); it makes the atomics of the deposit and the loads of the
// gather coherent again once clustering has scattered the initial
// (Lagrangian) order: neighbouring lanes of a warp then share cells and
// cache lines.
#include <algorithm>

#include "pm_kernels.cuh"

namespace pm {

namespace {
constexpr int RS_T = 256;                 // threads per tile
constexpr int RS_ITEMS = 16;              // keys per thread
constexpr int RS_TILE = RS_T * RS_ITEMS;  // 4096 keys per tile
constexpr int RS_BINS = 256;              // 8-bit digits
constexpr int RS_WARPS = RS_T / 32;
constexpr int RS_MAXPASS = 4;             // 30-bit keys (n_mesh <= 1024)
constexpr unsigned FULL = 0xffffffffu;

// cell of the CIC base node floor(u - 1/2) along each axis, wrapped into
// [0, n); a non-finite coordinate maps to 0
__device__ __forceinline__ unsigned cell_axis(float u, int n) {
  const float f = floorf(__fsub_rn(u, 0.5f));
  int i = (f >= -1.0e9f && f <= 1.0e9f) ? (int)f : 0;
  i %= n;
  if (i < 0) i += n;
  return (unsigned)i;
}
__device__ __forceinline__ unsigned cell_key(const float4& x, int n) {
  return (cell_axis(x.z, n) * (unsigned)n + cell_axis(x.y, n)) * (unsigned)n +
         cell_axis(x.x, n);
}

// add 1 to h[digit] for every valid lane, one shared atomic per distinct
// digit of the warp
__device__ __forceinline__ void warp_count(unsigned* h, unsigned dg, bool ok) {
  const int lane = threadIdx.x & 31;
  const unsigned peers = __match_any_sync(FULL, ok ? dg : 256u + lane);
  if (ok && lane == __ffs(peers) - 1) atomicAdd(h + dg, (unsigned)__popc(peers));
}
}  // namespace

// keys and identity values of one tile; the tile's counts of digit 0 into
// counts[d * T + tile], and every pass's digit totals into ghist
__global__ void __launch_bounds__(RS_T) k_sort_keys(const float4* __restrict__ pos, long long N,
                                                    int n, int npass,
                                                    unsigned* __restrict__ keys,
                                                    unsigned* __restrict__ vals,
                                                    unsigned* __restrict__ counts, int T,
                                                    unsigned* __restrict__ ghist) {
  __shared__ unsigned h[RS_MAXPASS * RS_BINS];
  for (int i = threadIdx.x; i < RS_MAXPASS * RS_BINS; i += RS_T) h[i] = 0u;
  __syncthreads();
  const long long base = (long long)blockIdx.x * RS_TILE;
  for (int r = 0; r < RS_ITEMS; ++r) {
    const long long i = base + (long long)r * RS_T + threadIdx.x;
    const bool ok = i < N;
    unsigned k = 0u;
    if (ok) {
      k = cell_key(pos[i], n);
      keys[i] = k;
      vals[i] = (unsigned)i;
    }
    for (int p = 0; p < npass; ++p) warp_count(h + p * RS_BINS, (k >> (8 * p)) & 255u, ok);
  }
  __syncthreads();
  const int d = threadIdx.x;
  counts[(size_t)d * T + blockIdx.x] = h[d];
  for (int p = 0; p < npass; ++p) {
    const unsigned c = h[p * RS_BINS + d];
    if (c) atomicAdd(ghist + p * RS_BINS + d, c);
  }
}

// the tile's counts of the digit at `shift`
__global__ void __launch_bounds__(RS_T) k_radix_hist(const unsigned* __restrict__ keys, long long N,
                                                     int shift, unsigned* __restrict__ counts,
                                                     int T) {
  __shared__ unsigned h[RS_BINS];
  h[threadIdx.x] = 0u;
  __syncthreads();
  const long long base = (long long)blockIdx.x * RS_TILE;
  for (int r = 0; r < RS_ITEMS; ++r) {
    const long long i = base + (long long)r * RS_T + threadIdx.x;
    const bool ok = i < N;
    const unsigned k = ok ? keys[i] : 0u;
    warp_count(h, (k >> shift) & 255u, ok);
  }
  __syncthreads();
  counts[(size_t)threadIdx.x * T + blockIdx.x] = h[threadIdx.x];
}

// block d: counts[d * T + t] <- number of keys with a smaller digit, plus
// those of digit d in tiles before t (the first destination of the tile's
// digit-d keys)
__global__ void __launch_bounds__(RS_T) k_radix_scan(unsigned* __restrict__ counts, int T,
                                                     const unsigned* __restrict__ gh) {
  __shared__ unsigned ws[RS_WARPS];
  __shared__ unsigned dbase;
  const int d = blockIdx.x, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  unsigned v = tid < d ? gh[tid] : 0u;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  if (lane == 0) ws[w] = v;
  __syncthreads();
  if (tid == 0) {
    unsigned b = 0u;
    for (int q = 0; q < RS_WARPS; ++q) b += ws[q];
    dbase = b;
  }
  __syncthreads();
  unsigned run = dbase;
  unsigned* c = counts + (size_t)d * T;
  for (int t0 = 0; t0 < T; t0 += RS_T) {
    const int t = t0 + tid;
    const unsigned x = t < T ? c[t] : 0u;
    unsigned inc = x;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(FULL, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane == 31) ws[w] = inc;
    __syncthreads();
    unsigned before = 0u, tot = 0u;
    for (int q = 0; q < RS_WARPS; ++q) {
      const unsigned s = ws[q];
      if (q < w) before += s;
      tot += s;
    }
    if (t < T) c[t] = run + before + inc - x;
    run += tot;
    __syncthreads();
  }
}

// stable scatter of one tile by the digit at `shift`: warp w takes keys
// [tile + 512 w, tile + 512 (w+1)) in rounds of 32; a key's destination is
// the tile's first slot of its digit + the keys of that digit in earlier
// warps + those earlier in its own warp
__global__ void __launch_bounds__(RS_T) k_radix_scatter(const unsigned* __restrict__ kin,
                                                        const unsigned* __restrict__ vin,
                                                        long long N, int shift,
                                                        const unsigned* __restrict__ offs, int T,
                                                        unsigned* __restrict__ kout,
                                                        unsigned* __restrict__ vout) {
  __shared__ unsigned wc[RS_WARPS * RS_BINS];
  __shared__ unsigned dbase[RS_BINS];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  for (int i = tid; i < RS_WARPS * RS_BINS; i += RS_T) wc[i] = 0u;
  dbase[tid] = offs[(size_t)tid * T + blockIdx.x];
  __syncthreads();
  unsigned* mine = wc + w * RS_BINS;
  const long long base = (long long)blockIdx.x * RS_TILE + (long long)w * (RS_ITEMS * 32);
  const unsigned lt = (1u << lane) - 1u;
  unsigned key[RS_ITEMS], val[RS_ITEMS], rank[RS_ITEMS];
#pragma unroll
  for (int r = 0; r < RS_ITEMS; ++r) {
    const long long i = base + r * 32 + lane;
    const bool ok = i < N;
    key[r] = ok ? kin[i] : 0u;
    val[r] = ok ? vin[i] : 0u;
    const unsigned dg = (key[r] >> shift) & 255u;
    const unsigned peers = __match_any_sync(FULL, ok ? dg : 256u + lane);
    const unsigned before = mine[dg];
    rank[r] = before + __popc(peers & lt);
    __syncwarp();
    if (ok && (peers >> lane) == 1u) mine[dg] = before + __popc(peers);  // last of its group
    __syncwarp();
  }
  __syncthreads();
  {
    unsigned run = 0u;
    for (int q = 0; q < RS_WARPS; ++q) {
      const unsigned c = wc[q * RS_BINS + tid];
      wc[q * RS_BINS + tid] = run;
      run += c;
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < RS_ITEMS; ++r) {
    const long long i = base + r * 32 + lane;
    if (i < N) {
      const unsigned dg = (key[r] >> shift) & 255u;
      const unsigned dst = dbase[dg] + mine[dg] + rank[r];
      if (dst < N) {  // always, the counts being those of the same keys
        kout[dst] = key[r];
        vout[dst] = val[r];
      }
    }
  }
}

__global__ void __launch_bounds__(256) k_permute(const float4* __restrict__ pos,
                                                 const float4* __restrict__ mom,
                                                 const unsigned* __restrict__ perm, long long N,
                                                 float4* __restrict__ pos_out,
                                                 float4* __restrict__ mom_out) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const unsigned j = perm[i];
    if (j >= N) continue;  // never: perm is a permutation of [0, N)
    pos_out[i] = pos[j];
    if (mom) mom_out[i] = mom[j];
  }
}

int sort_passes(int n) {
  unsigned long long m = (unsigned long long)n * n * n - 1ull;
  int bits = 0;
  while (m) {
    ++bits;
    m >>= 1;
  }
  return std::max(1, (bits + 7) / 8);
}

size_t sort_counts_len(long long N) {
  return (size_t)RS_BINS * (size_t)((N + RS_TILE - 1) / RS_TILE);
}

size_t sort_ghist_len() { return (size_t)RS_MAXPASS * RS_BINS; }

cudaError_t launch_sort_particles(cudaStream_t st, const float4* pos, const float4* mom,
                                  long long N, int n, const SortWork& w, float4* pos_out,
                                  float4* mom_out) {
  if (N <= 0) return cudaSuccess;
  const int T = (int)((N + RS_TILE - 1) / RS_TILE);
  const int np = sort_passes(n);
  cudaError_t e = cudaMemsetAsync(w.ghist, 0, sizeof(unsigned) * sort_ghist_len(), st);
  if (e != cudaSuccess) return e;
  k_sort_keys<<<T, RS_T, 0, st>>>(pos, N, n, np, w.keys[0], w.vals[0], w.counts, T, w.ghist);
  note_launch();
  int cur = 0;
  for (int p = 0; p < np; ++p) {
    if (p > 0) {
      k_radix_hist<<<T, RS_T, 0, st>>>(w.keys[cur], N, 8 * p, w.counts, T);
      note_launch();
    }
    k_radix_scan<<<RS_BINS, RS_T, 0, st>>>(w.counts, T, w.ghist + p * RS_BINS);
    note_launch();
    k_radix_scatter<<<T, RS_T, 0, st>>>(w.keys[cur], w.vals[cur], N, 8 * p, w.counts, T,
                                        w.keys[cur ^ 1], w.vals[cur ^ 1]);
    note_launch();
    cur ^= 1;
  }
  const int grid = (int)std::min<long long>((N + 255) / 256, 152LL * 16);
  k_permute<<<grid, 256, 0, st>>>(pos, mom, w.vals[cur], N, pos_out, mom_out);
  note_launch();
  return cudaGetLastError();
}

}  // namespace pm
