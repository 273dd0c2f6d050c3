// The forward 3x3x3 "same" convolution of the learned guess as an implicit
// GEMM on the 5th-generation tensor cores without an im2col copy.
//
// A CTA computes a T^3 block of output voxels of one sample.  It stages the
// (T+2)^3 input block once in shared memory, channel-blocked: block c holds
// channels 8c .. 8c+7 of every position as one 16-byte row, positions in
// raster order of the padded block (x fastest).  In the K-major no-swizzle
// canonical layout an MMA operand of 128 rows x 16 K-elements is two
// 8-element core-matrix columns, each 128 rows of 16 bytes at a common row
// stride of 16 bytes; so the A operand of tap (dz, dy, dx) for 128
// consecutive positions is the staged block itself, started
// ((dz-1) P_yx + (dy-1) P_x + (dx-1)) rows further on, with the second core
// column one channel block further (LBO = the block stride), or, for 8
// input channels, at the next tap (LBO = that tap's extra shift).  Every
// (tap, channel pair) is one tcgen05.mma issued straight from the staged
// input; the positions of a 128-row M tile that fall on the block's halo
// or outside the sample are computed and discarded.  All M tiles of the
// block accumulate in tensor memory at once; one commit, one bounded wait,
// then the epilogue (bias, ReLU, BF16 / FP32) reads TMEM row by row.
//
// Weights: wf [N][K] BF16, K = 28 taps x 8 (8 input channels: taps in pairs,
// the 28th zero) or 27 taps x cinp (cinp = cin rounded up to 16; channels
// beyond cin zero), tap-major, loaded whole into shared memory.
#include <cuda_bf16.h>

#include "pm_kernels.cuh"
#include "tc_gemm.cuh"

namespace pm {

namespace {

using bf16 = __nv_bfloat16;
constexpr long long CF_WAIT_LIMIT = 20000000;  // mbarrier polls before giving up
constexpr int CF_NT = 128;                     // threads per CTA (one per TMEM lane)
constexpr int CF_SLACK = 128;                  // rows past a block's end an M tile may touch
constexpr int CF_MAXK = 192;                   // K slices of 16 a layer may have

// q = x / d, r = x % d for 0 <= x < 2^22, 1 <= d <= 4096, from a float
// reciprocal (its error is below one, so one correction step suffices)
__device__ __forceinline__ void cf_divmod(int x, int d, float inv_d, int& q, int& r) {
  q = (int)((float)x * inv_d);
  r = x - q * d;
  if (r < 0) { --q; r += d; }
  else if (r >= d) { ++q; r -= d; }
}

// 16-byte asynchronous copy global -> shared; src_bytes 0 fills zeros
__device__ __forceinline__ void cf_cp16(uint8_t* smem, const void* gmem, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(tc::smem_u32(smem)),
               "l"(gmem), "r"(src_bytes)
               : "memory");
}

struct CfShape {
  int T;      // output block side
  int P;      // positions of the padded block, (T + 2)^3
  int nbr;    // channel blocks staged (cin / 8)
  int cbs;    // bytes between channel blocks (P + slack rows)
  int mt;     // M tiles of 128 positions
  int p0;     // position of the first output, (P_x + 1) P_x + 1 with P_x = T + 2
  int kf;     // K of wf
  int ncols;  // TMEM columns allocated (power of two >= mt N)
  int smem;   // dynamic shared memory bytes
};

__host__ __device__ inline CfShape cf_shape(int T, int cin, int n) {
  CfShape s{};
  const int px = T + 2;
  s.T = T;
  s.P = px * px * px;
  s.nbr = cin / 8;
  s.cbs = (s.P + CF_SLACK) * 16;
  s.p0 = (px + 1) * px + 1;
  const int last = (T * px + T) * px + T;  // position of the last output
  s.mt = (last - s.p0 + 1 + 127) / 128;
  s.kf = cin == 8 ? 28 * 8 : 27 * ((cin + 15) / 16 * 16);
  int need = s.mt * n, c = 32;
  while (c < need) c *= 2;
  s.ncols = c;
  s.smem = s.nbr * s.cbs + n * s.kf * 2 + 1024;
  return s;
}

template <int N>
__global__ void __launch_bounds__(CF_NT) k_conv_fast(const bf16* __restrict__ in, int B, int S,
                                                     int per, int cin,
                                                     const bf16* __restrict__ wf, CfShape sh,
                                                     const float* __restrict__ bias, int cout,
                                                     int relu, bf16* __restrict__ out_bf,
                                                     float* __restrict__ out_f, int* err) {
  extern __shared__ __align__(1024) uint8_t cf_sm[];
  __shared__ uint32_t tslot;
  __shared__ __align__(8) uint64_t mbar_s;
  // the A and B descriptors of every K slice for the first M tile (the
  // next tiles start 128 rows, i.e. 2048 bytes = 128 descriptor units, on)
  __shared__ uint64_t adesc[CF_MAXK], bdesc[CF_MAXK];
  // 1 KB-aligned start of the staged input; the weights follow the blocks
  uint8_t* sA = cf_sm + ((1024 - (tc::smem_u32(cf_sm) & 1023)) & 1023);
  uint8_t* sB = sA + sh.nbr * sh.cbs;
  const int T = sh.T, px = T + 2;
  const int tiles = (S + T - 1) / T;
  int bid = blockIdx.x;
  const int tx = bid % tiles; bid /= tiles;
  const int ty = bid % tiles; bid /= tiles;
  const int tz = bid % tiles;
  const int smp = bid / tiles;
  const int x0 = tx * T - 1, y0 = ty * T - 1, z0 = tz * T - 1;  // sample coordinates of position 0
  const long long sbase = (long long)smp * S * S * S;

  if (threadIdx.x < 32) tc::tmem_alloc(&tslot, sh.ncols);
  const uint32_t mbar = tc::smem_u32(&mbar_s);
  if (threadIdx.x == 0) tc::mbar_init(mbar, 1);

  // weights: row n, 16-byte group g of K in the canonical layout
  const int kg = sh.kf / 8;
  for (int t = threadIdx.x; t < N * kg; t += CF_NT) {
    const int n = t / kg, g = t - n * kg;
    *reinterpret_cast<uint4*>(sB + (n >> 3) * (sh.kf * 16) + g * 128 + (n & 7) * 16) =
        *reinterpret_cast<const uint4*>(wf + (long long)n * sh.kf + 8 * g);
  }
  // the padded input block, channel-blocked, by asynchronous 16-byte copies
  // (zero-filled outside an open sample, wrapped in a periodic one); the
  // slack rows are zeroed
  const int rows = sh.nbr * sh.P;
  const float inv_px = 1.0f / (float)px, inv_p = 1.0f / (float)sh.P;
  for (int t = threadIdx.x; t < rows; t += CF_NT) {
    int c, p, x, y, z, r;
    cf_divmod(t, sh.P, inv_p, c, p);
    cf_divmod(p, px, inv_px, r, x);
    cf_divmod(r, px, inv_px, z, y);
    int gx = x0 + x, gy = y0 + y, gz = z0 + z;
    if (per) {
      gx = gx < 0 ? gx + S : (gx >= S ? gx - S : gx);
      gy = gy < 0 ? gy + S : (gy >= S ? gy - S : gy);
      gz = gz < 0 ? gz + S : (gz >= S ? gz - S : gz);
    }
    const bool inside = gx >= 0 && gx < S && gy >= 0 && gy < S && gz >= 0 && gz < S;
    const long long vx = inside ? sbase + ((long long)gz * S + gy) * S + gx : 0;
    cf_cp16(sA + c * sh.cbs + p * 16, in + vx * cin + 8 * c, inside ? 16 : 0);
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
  for (int t = threadIdx.x; t < sh.nbr * CF_SLACK; t += CF_NT) {
    const int c = t / CF_SLACK, r = t - c * CF_SLACK;
    *reinterpret_cast<uint4*>(sA + c * sh.cbs + (sh.P + r) * 16) = make_uint4(0, 0, 0, 0);
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  const int nk = sh.kf / 16;  // MMAs per M tile
  {
    const uint32_t a0 = tc::smem_u32(sA), b0 = tc::smem_u32(sB);
    const uint32_t sbo_b = (uint32_t)sh.kf * 16u;
    const int cinp = cin == 8 ? 8 : (cin + 15) / 16 * 16;
    for (int s = threadIdx.x; s < nk; s += CF_NT) {
      uint32_t a, lbo;
      if (cin == 8) {
        // taps 2s and 2s + 1 (the 28th tap has zero weights: any rows)
        const int t0 = 2 * s, t1 = 2 * s + 1;
        const int sh0 = (t0 / 9 - 1) * px * px + ((t0 / 3) % 3 - 1) * px + (t0 % 3 - 1);
        const int sh1 = t1 < 27 ? (t1 / 9 - 1) * px * px + ((t1 / 3) % 3 - 1) * px + (t1 % 3 - 1)
                                : sh0;
        a = a0 + (uint32_t)(sh.p0 + sh0) * 16u;
        lbo = (uint32_t)(sh1 - sh0) * 16u;
      } else {
        // tap s / (cinp / 16), channel blocks 2j and 2j + 1 (a block past the
        // staged ones has zero weights: it re-reads block 2j)
        const int per_tap = cinp / 16;
        const int t = s / per_tap, j = s - t * per_tap;
        const int sht = (t / 9 - 1) * px * px + ((t / 3) % 3 - 1) * px + (t % 3 - 1);
        a = a0 + (uint32_t)(2 * j) * (uint32_t)sh.cbs + (uint32_t)(sh.p0 + sht) * 16u;
        lbo = 2 * j + 1 < sh.nbr ? (uint32_t)sh.cbs : 0u;
      }
      adesc[s] = tc::smem_desc(a, lbo, 128u);
      bdesc[s] = tc::smem_desc(b0 + 256u * (uint32_t)s, 128u, sbo_b);
    }
  }
  tc::fence_async_smem();
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t taddr = tslot;

  if (threadIdx.x == 0) {
    constexpr uint32_t IDESC = tc::idesc_bf16(tc::TM, N);
    for (int m = 0; m < sh.mt; ++m) {
      const uint64_t step = (uint64_t)(128 * m);  // 128 rows of 16 bytes, in 16-byte units
      for (int s = 0; s < nk; ++s)
        tc::mma_bf16(taddr + (uint32_t)(m * N), adesc[s] + step, bdesc[s], IDESC,
                     s > 0 ? 1u : 0u);
    }
    tc::mma_commit(mbar);
  }
  // the block decides together whether the MMAs completed
  const bool ok = __syncthreads_and(tc::mbar_wait(mbar, 0u, CF_WAIT_LIMIT)) != 0;
  if (!ok) {
    if (threadIdx.x == 0) atomicOr(err, 1);
    tc::mbar_wait(mbar, 0u, CF_WAIT_LIMIT);  // one more bounded wait before leaving
  } else {
    tc::tc_fence_after();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int coutp = (cout + 7) & ~7;
    for (int m = 0; m < sh.mt; ++m) {
      const int p = sh.p0 + 128 * m + 32 * w + lane;
      int x, y, z, r;
      cf_divmod(p, px, 1.0f / (float)px, r, x);
      cf_divmod(r, px, 1.0f / (float)px, z, y);
      const int gx = x0 + x, gy = y0 + y, gz = z0 + z;
      const bool valid = x >= 1 && x <= T && y >= 1 && y <= T && z >= 1 && z <= T &&
                         gx < S && gy < S && gz < S;
      const long long row = sbase + ((long long)gz * S + gy) * S + gx;
#pragma unroll
      for (int col = 0; col < N; col += 8) {
        float val[8];
        tc::tmem_ld8(taddr, w, m * N + col, val);
        if (valid && col < coutp) {
          __align__(16) bf16 ob[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            float o = col + q < cout ? val[q] + (bias ? bias[col + q] : 0.0f) : 0.0f;
            if (relu) o = fmaxf(o, 0.0f);
            ob[q] = __float2bfloat16_rn(o);
            if (out_f) out_f[row * coutp + col + q] = o;
          }
          if (out_bf)
            *reinterpret_cast<uint4*>(out_bf + row * coutp + col) =
                *reinterpret_cast<const uint4*>(ob);
        }
      }
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (threadIdx.x < 32) tc::tmem_free(taddr, sh.ncols);
}

// wf[n][k] from the FP32 masters w[co][tap * cin + ci] (see the file head)
__global__ void k_pack_wf(const float* __restrict__ w, int cin, int cout, int n, int kf,
                          bf16* __restrict__ wf) {
  const int cinp = cin == 8 ? 8 : (cin + 15) / 16 * 16;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n * kf; t += gridDim.x * blockDim.x) {
    const int r = t / kf, k = t - r * kf;
    const int tap = k / cinp, ci = k - tap * cinp;
    float v = 0.0f;
    if (r < cout && tap < 27 && ci < cin) v = w[(long long)r * 27 * cin + tap * cin + ci];
    wf[t] = __float2bfloat16_rn(v);
  }
}

constexpr int CF_SMEM_MAX = 200 * 1024;

template <int N>
bool cf_set_attr(int smem) {
  return cudaFuncSetAttribute(k_conv_fast<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              smem) == cudaSuccess;
}

}  // namespace

int conv_fast_kf(int cin);

// The block side for a layer, or 0 when the staged block and the weights do
// not fit in shared memory or the accumulators in 128 TMEM columns (four
// CTAs per SM) at any side >= 4.
int conv_fast_side(int cin, int cout) {
  if (cin % 8 != 0 || conv_fast_kf(cin) / 16 > CF_MAXK) return 0;
  const int n = cout <= 16 ? 16 : (cout + 15) / 16 * 16;
  if (n != 16 && n != 32 && n != 48 && n != 64) return 0;
  for (int T = 14; T >= 4; --T) {
    const CfShape s = cf_shape(T, cin, n);
    if (s.smem <= CF_SMEM_MAX && s.mt * n <= 128) return T;
  }
  return 0;
}

int conv_fast_kf(int cin) { return cin == 8 ? 28 * 8 : 27 * ((cin + 15) / 16 * 16); }

void launch_pack_wf(cudaStream_t st, const float* w, int cin, int cout, int n, void* wf) {
  const int kf = conv_fast_kf(cin);
  k_pack_wf<<<(n * kf + 255) / 256, 256, 0, st>>>(w, cin, cout, n, kf, (bf16*)wf);
  note_launch();
}

bool launch_conv_fast(cudaStream_t st, const void* in, int B, int S, int per, int cin,
                      const void* wf, int n, int T, const float* bias, int cout, int relu,
                      void* out_bf, float* out_f, int* err) {
  if (T > S) T = S;  // a block never larger than the sample
  const CfShape sh = cf_shape(T, cin, n);
  const int tiles = (S + T - 1) / T;
  const dim3 grid((unsigned)(B * tiles * tiles * tiles));
#define PM_CF(NN)                                                                       \
  if (!cf_set_attr<NN>(sh.smem)) return false;                                          \
  k_conv_fast<NN><<<grid, CF_NT, sh.smem, st>>>((const bf16*)in, B, S, per, cin,          \
                                                 (const bf16*)wf, sh, bias, cout, relu,    \
                                                 (bf16*)out_bf, out_f, err)
  switch (n) {
    case 16: PM_CF(16); break;
    case 32: PM_CF(32); break;
    case 48: PM_CF(48); break;
    case 64: PM_CF(64); break;
    default: return false;
  }
#undef PM_CF
  note_launch();
  return true;
}

}  // namespace pm
