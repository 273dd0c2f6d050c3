// Particle-side kernels: gradient + CIC gather + kick + half drift + keep
// flag (Sec. 2.2, second and third DKD lines; Sec. 2.4 footnote: the gather
// uses the deposit's CIC weights), and the order-preserving compaction that
// drops particles leaving the lightcone (Sec. 2.4: active particles are
// recomputed at the end of every step; Table 2, last row).
#include "mg_arith.cuh"
#include "pm_kernels.cuh"

namespace pm {

constexpr int KCHUNK = PART_CHUNK;  // KT threads x KITEMS particles per block

// ---------------------------------------------------------------------------
// Gradient + CIC gather + kick + drift + keep flag.  For each particle: the
// CIC nodes (i, i+1 per axis; wrapped when periodic), the centred difference
// of Phi = hi + lo at each node, g = (hi(i+1) - hi(i-1)) + (lo(i+1) -
// lo(i-1)), weighted with (2^16 - dq, dq) / 2^16, then p -= kick grad(Phi),
// x = fl(x + fl(p c2)), and keep = x inside [klo, khi]^3 (exact float bounds
// of |x - c| <= R).  Block b covers particles [b KCHUNK, (b+1) KCHUNK) and
// writes its keep count.
//
// GF: the node differences come from the gradient field G (k_grad, one
// float4 per mesh cell: 8 loads per particle) instead of from Phi (32 mesh
// points, hi and lo: 64 loads).  Both forms apply the same operations in the
// same order, so they give the same bits.
// ---------------------------------------------------------------------------
// F += wa wb (w0 g0 + w1 g1)
__device__ __forceinline__ float cic_acc(float F, float wa, float wb, float w0, float g0,
                                         float w1, float g1) {
  const float inner = __fmaf_rn(w1, g1, __fmul_rn(w0, g0));
  return __fmaf_rn(__fmul_rn(wa, wb), inner, F);
}

template <bool GF>
__device__ __forceinline__ void d_gather_kick_drift(const BI& bi,
    float4* __restrict__ pos, float4* __restrict__ mom, long long N,
    const float* __restrict__ ph, const float* __restrict__ pl,
    const float4* __restrict__ G, int n, int lo, int s,
    int periodic, float kick, float c2, int do_flag, float klo, float khi, KeepBall kb,
    unsigned char* __restrict__ flags, unsigned int* __restrict__ block_keep,
    float4* __restrict__ forces, unsigned long long* __restrict__ escaped){
  const int P = n + 2;
  const float fn = (float)n;
  const long long base = (long long)bi.x * KCHUNK;
  unsigned int keep_count = 0, esc = 0;
#pragma unroll 1
  for (int it = 0; it < KITEMS; ++it) {
    long long p = base + it * KT + threadIdx.x;
    if (p >= N) break;
    float4 x = pos[p];
    float4 v = mom[p];
    int ix, iy, iz, dx, dy, dz;
    cic_axis(x.x, ix, dx);
    cic_axis(x.y, iy, dy);
    cic_axis(x.z, iz, dz);
    float Fx = 0.f, Fy = 0.f, Fz = 0.f;
    bool ok = true;
    int X[4], Y[4], Z[4];
    if (periodic) {
      ok = !(ix < -1 || ix > n - 1 || iy < -1 || iy > n - 1 || iz < -1 || iz > n - 1);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        int a = ix - 1 + q, b = iy - 1 + q, c = iz - 1 + q;
        X[q] = ok ? (a < 0 ? a + n : (a >= n ? a - n : a)) : 0;
        Y[q] = ok ? (b < 0 ? b + n : (b >= n ? b - n : b)) : 0;
        Z[q] = ok ? (c < 0 ? c + n : (c >= n ? c - n : c)) : 0;
      }
    } else {
      const int hi = lo + s - 1;
      ok = !(ix < lo || ix + 1 > hi || iy < lo || iy + 1 > hi || iz < lo || iz + 1 > hi);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        X[q] = ok ? ix - 1 + q : lo;
        Y[q] = ok ? iy - 1 + q : lo;
        Z[q] = ok ? iz - 1 + q : lo;
      }
    }
    if (ok) {
      const float sc = 1.0f / 65536.0f;
      const float wx[2] = {(float)(65536 - dx) * sc, (float)dx * sc};
      const float wy[2] = {(float)(65536 - dy) * sc, (float)dy * sc};
      const float wz[2] = {(float)(65536 - dz) * sc, (float)dz * sc};
      int RY[4], RZ[4], CX[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        RY[q] = (Y[q] + 1) * P;
        RZ[q] = (Z[q] + 1) * P * P;
        CX[q] = X[q] + 1;
      }
      // gx/gy/gz[c][b][a]: the centred differences at node (X[a+1], Y[b+1], Z[c+1])
      float gx[2][2][2], gy[2][2][2], gz[2][2][2];
      if (GF) {
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
          for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int a = 0; a < 2; ++a) {
              const float4 g = __ldg(G + RZ[c + 1] + RY[b + 1] + CX[a + 1]);
              gx[c][b][a] = g.x;
              gy[c][b][a] = g.y;
              gz[c][b][a] = g.z;
            }
      } else {
        // the 8 nodes' centred differences touch 32 distinct mesh points:
        // the 16 of the x-rows (y, z in the node range), plus 8 more in y
        // and 8 in z; each is loaded once (hi and lo)
        float Hx[2][2][4], Lx[2][2][4];  // [c][b][q]: (X[q], Y[b+1], Z[c+1])
        float Hy[2][2][2], Ly[2][2][2];  // [c][a][e]: (X[a+1], Y[3e], Z[c+1])
        float Hz[2][2][2], Lz[2][2][2];  // [b][a][e]: (X[a+1], Y[b+1], Z[3e])
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
          for (int b = 0; b < 2; ++b) {
            int r = RZ[c + 1] + RY[b + 1];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              Hx[c][b][q] = ph[r + CX[q]];
              Lx[c][b][q] = pl[r + CX[q]];
            }
          }
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
          for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int e = 0; e < 2; ++e) {
              int r = RZ[c + 1] + RY[3 * e] + CX[a + 1];
              Hy[c][a][e] = ph[r];
              Ly[c][a][e] = pl[r];
            }
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
          for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int e = 0; e < 2; ++e) {
              int r = RZ[3 * e] + RY[b + 1] + CX[a + 1];
              Hz[b][a][e] = ph[r];
              Lz[b][a][e] = pl[r];
            }
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
          for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int a = 0; a < 2; ++a) {
              gx[c][b][a] = gdiff(Hx[c][b][a + 2], Hx[c][b][a], Lx[c][b][a + 2], Lx[c][b][a]);
              // y: node Y[b+1] takes Y[b+2] - Y[b]
              const float yp = b == 0 ? Hx[c][1][a + 1] : Hy[c][a][1];
              const float ym = b == 0 ? Hy[c][a][0] : Hx[c][0][a + 1];
              const float lyp = b == 0 ? Lx[c][1][a + 1] : Ly[c][a][1];
              const float lym = b == 0 ? Ly[c][a][0] : Lx[c][0][a + 1];
              gy[c][b][a] = gdiff(yp, ym, lyp, lym);
              const float zp = c == 0 ? Hx[1][b][a + 1] : Hz[b][a][1];
              const float zm = c == 0 ? Hz[b][a][0] : Hx[0][b][a + 1];
              const float lzp = c == 0 ? Lx[1][b][a + 1] : Lz[b][a][1];
              const float lzm = c == 0 ? Lz[b][a][0] : Lx[0][b][a + 1];
              gz[c][b][a] = gdiff(zp, zm, lzp, lzm);
            }
      }
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int b = 0; b < 2; ++b)
          Fx = cic_acc(Fx, wy[b], wz[c], wx[0], gx[c][b][0], wx[1], gx[c][b][1]);
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int a = 0; a < 2; ++a)
          Fy = cic_acc(Fy, wx[a], wz[c], wy[0], gy[c][0][a], wy[1], gy[c][1][a]);
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int a = 0; a < 2; ++a)
          Fz = cic_acc(Fz, wx[a], wy[b], wz[0], gz[0][b][a], wz[1], gz[1][b][a]);
      Fx = __fmul_rn(Fx, 0.5f);
      Fy = __fmul_rn(Fy, 0.5f);
      Fz = __fmul_rn(Fz, 0.5f);
    } else {
      ++esc;
    }
    v.x = __fmaf_rn(-kick, Fx, v.x);
    v.y = __fmaf_rn(-kick, Fy, v.y);
    v.z = __fmaf_rn(-kick, Fz, v.z);
    x.x = __fadd_rn(x.x, __fmul_rn(v.x, c2));
    x.y = __fadd_rn(x.y, __fmul_rn(v.y, c2));
    x.z = __fadd_rn(x.z, __fmul_rn(v.z, c2));
    if (periodic) {
      if (x.x < 0.f) x.x = __fadd_rn(x.x, fn);
      if (x.x >= fn) x.x = __fsub_rn(x.x, fn);
      if (x.y < 0.f) x.y = __fadd_rn(x.y, fn);
      if (x.y >= fn) x.y = __fsub_rn(x.y, fn);
      if (x.z < 0.f) x.z = __fadd_rn(x.z, fn);
      if (x.z >= fn) x.z = __fsub_rn(x.z, fn);
    }
    pos[p] = x;
    mom[p] = v;
    if (forces) forces[p] = make_float4(Fx, Fy, Fz, 0.f);
    if (do_flag) {
      const bool keep = in_keep(x, klo, khi, kb);
      flags[p] = keep ? 1 : 0;
      keep_count += keep ? 1u : 0u;
    }
  }
  if (do_flag) {
    __shared__ unsigned int sk[KT / 32];
    unsigned int w = keep_count;
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    if ((threadIdx.x & 31) == 0) sk[threadIdx.x >> 5] = w;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned int t = 0;
      for (int q = 0; q < KT / 32; ++q) t += sk[q];
      block_keep[bi.x] = t;
    }
  }
  {
    unsigned int w = esc;
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    if ((threadIdx.x & 31) == 0 && w) atomicAdd(escaped, (unsigned long long)w);
  }
}

template <bool GF>
__global__ void __launch_bounds__(KT) k_gather_kick_drift(
    float4* __restrict__ pos, float4* __restrict__ mom, long long N,
    const float* __restrict__ ph, const float* __restrict__ pl, const float4* __restrict__ G,
    int n, int lo, int s, int periodic, float kick, float c2, int do_flag, float klo, float khi,
    KeepBall kb, unsigned char* __restrict__ flags, unsigned int* __restrict__ block_keep,
    float4* __restrict__ forces, unsigned long long* __restrict__ escaped) {
  pdl_wait();
  pdl_release();
  d_gather_kick_drift<GF>(bi_native(), pos, mom, N, ph, pl, G, n, lo, s, periodic, kick, c2,
                          do_flag, klo, khi, kb, flags, block_keep, forces, escaped);
}

// G(c) = (gx, gy, gz, 0): centred differences of Phi = hi + lo at every cell
// of the active cube (wrapped when periodic, ghost values when open), in the
// full (n+2)^3 layout of Phi.
__global__ void __launch_bounds__(256) k_grad(const float* __restrict__ ph,
                                              const float* __restrict__ pl, int n, int lo,
                                              int s, int periodic, float4* __restrict__ G) {
  pdl_wait();
  pdl_release();
  d_grad(bi_native(), ph, pl, n, lo, s, periodic, G);
}

// ---------------------------------------------------------------------------
// TSC variant of the gather + kick + drift (+ keep flags): the node
// differences of G at the 27 TSC nodes with the deposit's Q16 weights
// (tsc_axis) scaled to float; same chunking as the CIC gather, so the keep
// counts feed the same scan.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void tsc_axis_f(float u, int& i, float w[3]) {
  const int iq = __float2int_rd(__fmul_rn(u, 65536.0f));
  i = iq >> 16;
  const unsigned long long q = (unsigned long long)(iq & 0xffff);
  const unsigned long long a = 65536ull - q;
  const unsigned int w0 = (unsigned int)((a * a) >> 17), w2 = (unsigned int)((q * q) >> 17);
  const float sc = 1.0f / 65536.0f;
  w[0] = (float)w0 * sc;
  w[1] = (float)(65536u - w0 - w2) * sc;
  w[2] = (float)w2 * sc;
}

__global__ void __launch_bounds__(KT) k_gather_tsc(
    float4* __restrict__ pos, float4* __restrict__ mom, long long N,
    const float4* __restrict__ G, int n, int lo, int s, int periodic, float kick, float c2,
    int do_flag, float klo, float khi, unsigned char* __restrict__ flags,
    unsigned int* __restrict__ block_keep, float4* __restrict__ forces,
    unsigned long long* __restrict__ escaped) {
  const int P = n + 2;
  const float fn = (float)n;
  const long long base = (long long)blockIdx.x * KCHUNK;
  unsigned int keep_count = 0, esc = 0;
#pragma unroll 1
  for (int it = 0; it < KITEMS; ++it) {
    const long long p = base + it * KT + threadIdx.x;
    if (p >= N) break;
    float4 x = pos[p];
    float4 v = mom[p];
    int i3[3];
    float w[3][3];
    tsc_axis_f(x.x, i3[0], w[0]);
    tsc_axis_f(x.y, i3[1], w[1]);
    tsc_axis_f(x.z, i3[2], w[2]);
    bool ok = true;
    int nd[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (periodic) {
        ok = ok && i3[a] >= 0 && i3[a] <= n - 1;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const int q = i3[a] - 1 + c;
          nd[a][c] = q < 0 ? q + n : (q >= n ? q - n : q);
        }
      } else {
        ok = ok && i3[a] - 1 >= lo && i3[a] + 1 <= lo + s - 1;
#pragma unroll
        for (int c = 0; c < 3; ++c) nd[a][c] = i3[a] - 1 + c;
      }
    }
    float Fx = 0.f, Fy = 0.f, Fz = 0.f;
    if (ok) {
#pragma unroll
      for (int cz = 0; cz < 3; ++cz)
#pragma unroll
        for (int cy = 0; cy < 3; ++cy) {
          const float wyz = __fmul_rn(w[1][cy], w[2][cz]);
          const long long row = ((long long)(nd[2][cz] + 1) * P + (nd[1][cy] + 1)) * P + 1;
#pragma unroll
          for (int cx = 0; cx < 3; ++cx) {
            const float4 g = __ldg(G + row + nd[0][cx]);
            const float wt = __fmul_rn(wyz, w[0][cx]);
            Fx = __fmaf_rn(wt, g.x, Fx);
            Fy = __fmaf_rn(wt, g.y, Fy);
            Fz = __fmaf_rn(wt, g.z, Fz);
          }
        }
      Fx = __fmul_rn(Fx, 0.5f);
      Fy = __fmul_rn(Fy, 0.5f);
      Fz = __fmul_rn(Fz, 0.5f);
    } else {
      ++esc;
    }
    v.x = __fmaf_rn(-kick, Fx, v.x);
    v.y = __fmaf_rn(-kick, Fy, v.y);
    v.z = __fmaf_rn(-kick, Fz, v.z);
    x.x = __fadd_rn(x.x, __fmul_rn(v.x, c2));
    x.y = __fadd_rn(x.y, __fmul_rn(v.y, c2));
    x.z = __fadd_rn(x.z, __fmul_rn(v.z, c2));
    if (periodic) {
      if (x.x < 0.f) x.x = __fadd_rn(x.x, fn);
      if (x.x >= fn) x.x = __fsub_rn(x.x, fn);
      if (x.y < 0.f) x.y = __fadd_rn(x.y, fn);
      if (x.y >= fn) x.y = __fsub_rn(x.y, fn);
      if (x.z < 0.f) x.z = __fadd_rn(x.z, fn);
      if (x.z >= fn) x.z = __fsub_rn(x.z, fn);
    }
    pos[p] = x;
    mom[p] = v;
    if (forces) forces[p] = make_float4(Fx, Fy, Fz, 0.f);
    if (do_flag) {
      const bool keep = x.x >= klo && x.x <= khi && x.y >= klo && x.y <= khi &&
                        x.z >= klo && x.z <= khi;
      flags[p] = keep ? 1 : 0;
      keep_count += keep ? 1u : 0u;
    }
  }
  if (do_flag) {
    __shared__ unsigned int sk[KT / 32];
    unsigned int wsum = keep_count;
    for (int o = 16; o > 0; o >>= 1) wsum += __shfl_xor_sync(0xffffffffu, wsum, o);
    if ((threadIdx.x & 31) == 0) sk[threadIdx.x >> 5] = wsum;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned int t = 0;
      for (int q = 0; q < KT / 32; ++q) t += sk[q];
      block_keep[blockIdx.x] = t;
    }
  }
  unsigned int we = esc;
  for (int o = 16; o > 0; o >>= 1) we += __shfl_xor_sync(0xffffffffu, we, o);
  if ((threadIdx.x & 31) == 0 && we) atomicAdd(escaped, (unsigned long long)we);
}

void launch_gather_tsc(cudaStream_t st, float4* pos, float4* mom, long long N,
                       const float4* G, int n, int lo, int s, int periodic, float kick,
                       float c2, int do_flag, float klo, float khi, unsigned char* flags,
                       unsigned int* block_keep, float4* forces,
                       unsigned long long* escaped) {
  if (N <= 0) return;
  k_gather_tsc<<<gkd_blocks(N), KT, 0, st>>>(pos, mom, N, G, n, lo, s, periodic, kick, c2,
                                             do_flag, klo, khi, flags, block_keep, forces,
                                             escaped);
  note_launch();
}

int gkd_blocks(long long N) { return (int)((N + KCHUNK - 1) / KCHUNK); }

void launch_gather_kick_drift(cudaStream_t st, float4* pos, float4* mom, long long N,
                              const float* ph, const float* pl, const float4* G, int n, int lo,
                              int s, int periodic, float kick, float c2, bool do_flag, float klo,
                              float khi, KeepBall kb, unsigned char* flags,
                              unsigned int* block_keep, float4* forces,
                              unsigned long long* escaped) {
  if (N <= 0) return;
  if (G)
    launch_pdl(k_gather_kick_drift<true>, dim3(gkd_blocks(N)), dim3(KT), 0, st, pos, mom, N, ph,
               pl, G, n, lo, s, periodic, kick, c2, do_flag ? 1 : 0, klo, khi, kb, flags,
               block_keep, forces, escaped);
  else
    launch_pdl(k_gather_kick_drift<false>, dim3(gkd_blocks(N)), dim3(KT), 0, st, pos, mom, N, ph,
               pl, G, n, lo, s, periodic, kick, c2, do_flag ? 1 : 0, klo, khi, kb, flags,
               block_keep, forces, escaped);
  note_launch();
}

void launch_grad(cudaStream_t st, const float* ph, const float* pl, int n, int lo, int s,
                 int periodic, float4* G) {
  dim3 grid((unsigned)((s + 31) / 32), (unsigned)((s + 7) / 8), (unsigned)s);
  launch_pdl(k_grad, grid, dim3(32, 8), 0, st, ph, pl, n, lo, s, periodic, G);
  note_launch();
}

// ---------------------------------------------------------------------------
// Keep flags from an explicit keep cube (pm_shrink), same chunking.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(KT) k_flag(const float4* __restrict__ pos, long long N,
                                             float klo, float khi, KeepBall kb,
                                             unsigned char* __restrict__ flags,
                                             unsigned int* __restrict__ block_keep) {
  const long long base = (long long)blockIdx.x * KCHUNK;
  unsigned int keep_count = 0;
  for (int it = 0; it < KITEMS; ++it) {
    long long p = base + it * KT + threadIdx.x;
    if (p >= N) break;
    const float4 x = pos[p];
    const bool keep = in_keep(x, klo, khi, kb);
    flags[p] = keep ? 1 : 0;
    keep_count += keep;
  }
  __shared__ unsigned int sk[KT / 32];
  unsigned int w = keep_count;
  for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
  if ((threadIdx.x & 31) == 0) sk[threadIdx.x >> 5] = w;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int t = 0;
    for (int q = 0; q < KT / 32; ++q) t += sk[q];
    block_keep[blockIdx.x] = t;
  }
}

void launch_flag(cudaStream_t st, const float4* pos, long long N, float klo, float khi,
                 unsigned char* flags, unsigned int* block_keep, KeepBall kb) {
  if (N <= 0) return;
  k_flag<<<gkd_blocks(N), KT, 0, st>>>(pos, N, klo, khi, kb, flags, block_keep);
  note_launch();
}

// ---------------------------------------------------------------------------
// Exclusive scan of the per-block keep counts (one CTA; nblk <= 2^24 at
// 1024 threads x 16k items), total written to *n_keep.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void d_scan_blocks(const BI& bi, const unsigned int* __restrict__ cnt,
                                                      unsigned long long* __restrict__ off,
                                                      int nblk,
                                                      unsigned long long* __restrict__ n_keep){
  __shared__ unsigned long long part[1024];
  const int tid = threadIdx.x;
  const int per = (nblk + 1023) / 1024;
  const int b0 = tid * per;
  unsigned long long s = 0;
  for (int q = 0; q < per; ++q) {
    int b = b0 + q;
    if (b < nblk) s += cnt[b];
  }
  part[tid] = s;
  __syncthreads();
  // Hillis-Steele inclusive scan over 1024 partials
  for (int o = 1; o < 1024; o <<= 1) {
    unsigned long long v = tid >= o ? part[tid - o] : 0ull;
    __syncthreads();
    part[tid] += v;
    __syncthreads();
  }
  unsigned long long run = tid ? part[tid - 1] : 0ull;
  for (int q = 0; q < per; ++q) {
    int b = b0 + q;
    if (b < nblk) {
      off[b] = run;
      run += cnt[b];
    }
  }
  if (tid == 1023) *n_keep = part[1023];
}

__global__ void __launch_bounds__(1024) k_scan_blocks(const unsigned int* __restrict__ cnt,
                                                      unsigned long long* __restrict__ off,
                                                      int nblk,
                                                      unsigned long long* __restrict__ n_keep) {
  d_scan_blocks(bi_native(), cnt, off, nblk, n_keep);
}

void launch_scan_blocks(cudaStream_t st, const unsigned int* cnt, unsigned long long* off,
                        int nblk, unsigned long long* n_keep) {
  k_scan_blocks<<<1, 1024, 0, st>>>(cnt, off, nblk, n_keep);
  note_launch();
}

// ---------------------------------------------------------------------------
// Stable scatter: survivors to out[keep_off[b] + rank], leavers to the
// lightcone at lc_base + (b*KCHUNK - keep_off[b]) + rank, both in index order.
// Leavers get mom.w = a_cross.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void d_scatter(const BI& bi, 
    const float4* __restrict__ pos, const float4* __restrict__ mom, long long N,
    const unsigned char* __restrict__ flags, const unsigned long long* __restrict__ keep_off,
    float4* __restrict__ pos_out, float4* __restrict__ mom_out, float4* __restrict__ lc_pos,
    float4* __restrict__ lc_mom, long long lc_base, float a_cross){
  __shared__ unsigned int wk[KT / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long base = (long long)bi.x * KCHUNK;
  unsigned long long keep_run = keep_off[bi.x];
  unsigned long long leave_run = (unsigned long long)base - keep_run;
  for (int it = 0; it < KITEMS; ++it) {
    long long p = base + it * KT + threadIdx.x;
    bool valid = p < N;
    bool keep = valid && flags[p];
    unsigned int bal = __ballot_sync(0xffffffffu, keep);
    unsigned int balv = __ballot_sync(0xffffffffu, valid);
    if (lane == 0) wk[warp] = __popc(bal);
    __syncthreads();
    unsigned int before = 0, row_keep = 0;
    for (int q = 0; q < KT / 32; ++q) {
      unsigned int c = wk[q];
      if (q < warp) before += c;
      row_keep += c;
    }
    unsigned int lanemask = (1u << lane) - 1u;
    unsigned int krank = before + __popc(bal & lanemask);
    // leavers before this lane in the row: valid lanes before minus keepers
    unsigned int vbefore = warp * 32 + __popc(balv & lanemask);
    unsigned int lrank = vbefore - krank;
    if (valid) {
      float4 x = pos[p], v = mom[p];
      if (keep) {
        unsigned long long d = keep_run + krank;
        pos_out[d] = x;
        mom_out[d] = v;
      } else {
        long long d = lc_base + (long long)(leave_run + lrank);
        v.w = a_cross;
        lc_pos[d] = x;
        lc_mom[d] = v;
      }
    }
    long long row_valid = N - (base + it * KT);
    row_valid = row_valid > KT ? KT : (row_valid < 0 ? 0 : row_valid);
    keep_run += row_keep;
    leave_run += (unsigned long long)row_valid - row_keep;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(KT) k_scatter(
    const float4* __restrict__ pos, const float4* __restrict__ mom, long long N,
    const unsigned char* __restrict__ flags, const unsigned long long* __restrict__ keep_off,
    float4* __restrict__ pos_out, float4* __restrict__ mom_out, float4* __restrict__ lc_pos,
    float4* __restrict__ lc_mom, long long lc_base, float a_cross) {
  d_scatter(bi_native(), pos, mom, N, flags, keep_off, pos_out, mom_out, lc_pos, lc_mom, lc_base, a_cross);
}

void launch_scatter(cudaStream_t st, const float4* pos, const float4* mom, long long N,
                    const unsigned char* flags, const unsigned long long* keep_off,
                    float4* pos_out, float4* mom_out, float4* lc_pos, float4* lc_mom,
                    long long lc_base, float a_cross) {
  if (N <= 0) return;
  k_scatter<<<gkd_blocks(N), KT, 0, st>>>(pos, mom, N, flags, keep_off, pos_out, mom_out,
                                          lc_pos, lc_mom, lc_base, a_cross);
  note_launch();
}

// ---------------------------------------------------------------------------
// Lightcone record without removal (fixed-box run): flag = outside the keep
// cube and not yet recorded (mom.w == 0); the flagged records are copied in
// index order to lc_base + off[b] + rank with mom.w = a_cross, and their
// mom.w in place is set to a_cross.  Nothing is written at or beyond lc_cap
// (the host compares the count with the capacity afterwards).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(KT) k_flag_record(const float4* __restrict__ pos,
                                                    const float4* __restrict__ mom, long long N,
                                                    float klo, float khi, KeepBall kb,
                                                    unsigned char* __restrict__ flags,
                                                    unsigned int* __restrict__ block_cnt) {
  const long long base = (long long)blockIdx.x * KCHUNK;
  unsigned int cnt = 0;
  for (int it = 0; it < KITEMS; ++it) {
    long long p = base + it * KT + threadIdx.x;
    if (p >= N) break;
    const float4 x = pos[p];
    const bool inside = in_keep(x, klo, khi, kb);
    const bool rec = !inside && mom[p].w == 0.0f;
    flags[p] = rec ? 1 : 0;
    cnt += rec ? 1u : 0u;
  }
  __shared__ unsigned int sk[KT / 32];
  unsigned int w = cnt;
  for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
  if ((threadIdx.x & 31) == 0) sk[threadIdx.x >> 5] = w;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int t = 0;
    for (int q = 0; q < KT / 32; ++q) t += sk[q];
    block_cnt[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(KT) k_record(const float4* __restrict__ pos,
                                               float4* __restrict__ mom, long long N,
                                               const unsigned char* __restrict__ flags,
                                               const unsigned long long* __restrict__ off,
                                               float4* __restrict__ lc_pos,
                                               float4* __restrict__ lc_mom, long long lc_base,
                                               long long lc_cap, float a_cross) {
  __shared__ unsigned int wk[KT / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long base = (long long)blockIdx.x * KCHUNK;
  unsigned long long run = off[blockIdx.x];
  for (int it = 0; it < KITEMS; ++it) {
    const long long p = base + it * KT + threadIdx.x;
    const bool rec = p < N && flags[p];
    const unsigned int bal = __ballot_sync(0xffffffffu, rec);
    if (lane == 0) wk[warp] = __popc(bal);
    __syncthreads();
    unsigned int before = 0, row = 0;
    for (int q = 0; q < KT / 32; ++q) {
      const unsigned int c = wk[q];
      if (q < warp) before += c;
      row += c;
    }
    const long long d = lc_base + (long long)(run + before + __popc(bal & ((1u << lane) - 1u)));
    if (rec && d < lc_cap) {
      float4 v = mom[p];
      v.w = a_cross;
      lc_pos[d] = pos[p];
      lc_mom[d] = v;
      mom[p].w = a_cross;
    }
    run += row;
    __syncthreads();
  }
}

void launch_flag_record(cudaStream_t st, const float4* pos, const float4* mom, long long N,
                        float klo, float khi, unsigned char* flags, unsigned int* block_cnt,
                        KeepBall kb) {
  if (N <= 0) return;
  k_flag_record<<<gkd_blocks(N), KT, 0, st>>>(pos, mom, N, klo, khi, kb, flags, block_cnt);
  note_launch();
}

void launch_record(cudaStream_t st, const float4* pos, float4* mom, long long N,
                   const unsigned char* flags, const unsigned long long* off, float4* lc_pos,
                   float4* lc_mom, long long lc_base, long long lc_cap, float a_cross) {
  if (N <= 0) return;
  k_record<<<gkd_blocks(N), KT, 0, st>>>(pos, mom, N, flags, off, lc_pos, lc_mom, lc_base,
                                         lc_cap, a_cross);
  note_launch();
}

// ---------------------------------------------------------------------------
// Batched forms.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) kb_grad(const GradDesc* d, const BTable* t) {
  int q;
  BI bi;
  if (!batch_map(d, t, (const int*)nullptr, q, bi)) return;
  const GradDesc& e = d[q];
  const bool alt = e.flip && (e.flip[e.r] & 1);
  d_grad(bi, alt ? e.ph_alt : e.ph, alt ? e.pl_alt : e.pl, e.n, e.lo, e.s, e.periodic, e.G);
}
__global__ void __launch_bounds__(KT) kb_gather(const GatherDesc* d, const BTable* t) {
  int q;
  BI bi;
  if (!batch_map(d, t, (const int*)nullptr, q, bi)) return;
  const GatherDesc& e = d[q];
  d_gather_kick_drift<true>(bi, e.pos, e.mom, e.N, nullptr, nullptr, e.G, e.n, e.lo, e.s,
                             e.periodic, e.kick, e.c2, e.do_flag, e.klo, e.khi,
                             KeepBall{0, 0.0, 0.0}, e.flags,
                             e.block_keep, e.forces, e.escaped);
}
__global__ void __launch_bounds__(1024) kb_scan(const ScanDesc* d, const BTable* t) {
  int q;
  BI bi;
  if (!batch_map(d, t, (const int*)nullptr, q, bi)) return;
  const ScanDesc& e = d[q];
  d_scan_blocks(bi, e.cnt, e.off, e.nblk, e.n_keep);
}
__global__ void __launch_bounds__(KT) kb_scatter(const ScatterDesc* d, const BTable* t) {
  int q;
  BI bi;
  if (!batch_map(d, t, (const int*)nullptr, q, bi)) return;
  const ScatterDesc& e = d[q];
  d_scatter(bi, e.pos, e.mom, e.N, e.flags, e.keep_off, e.pos_out, e.mom_out, e.lc_pos,
            e.lc_mom, e.lc_base, e.a_cross);
}

void launch_grad_b(cudaStream_t st, int grid, const GradDesc* d, const BTable* t) {
  if (grid <= 0) return;
  kb_grad<<<grid, dim3(32, 8), 0, st>>>(d, t);
  note_launch();
}
void launch_gather_b(cudaStream_t st, int grid, const GatherDesc* d, const BTable* t) {
  if (grid <= 0) return;
  kb_gather<<<grid, KT, 0, st>>>(d, t);
  note_launch();
}
void launch_scan_b(cudaStream_t st, int grid, const ScanDesc* d, const BTable* t) {
  if (grid <= 0) return;
  kb_scan<<<grid, 1024, 0, st>>>(d, t);
  note_launch();
}
void launch_scatter_b(cudaStream_t st, int grid, const ScatterDesc* d, const BTable* t) {
  if (grid <= 0) return;
  kb_scatter<<<grid, KT, 0, st>>>(d, t);
  note_launch();
}

}  // namespace pm
