// Mesh-side kernels of the PM step: fused half drift + fixed-point CIC
// deposit (Sec. 2.2 first DKD line; Sec. 2.4 footnote, CIC), the Poisson
// source on the active cube (Sec. 2.1, Eq. 3) with its boundary multipoles,
// and the open-boundary ghost layer (Table 1: open boundaries).
#include <algorithm>
#include <cooperative_groups.h>

#include "pm_kernels.cuh"

namespace cg = cooperative_groups;

namespace pm {

// ---------------------------------------------------------------------------
// K1: x += p * c0 (float32, two roundings), then the 8 int64 CIC weights.
// Periodic: nodes wrap mod n.  Open: a particle with a node outside the cube
// [lo, lo+s) deposits nothing and is counted as escaped.  The weights of
// lanes that share a cell, and the shared column of x-neighbouring cells,
// are summed within the warp first (integers: the same totals), so that a
// cell-ordered warp issues about one set of atomics per cell.
// ---------------------------------------------------------------------------
template <bool DRIFT>
__device__ __forceinline__ void d_drift_deposit(const BI& bi, 
    float4* __restrict__ pos, const float4* __restrict__ mom, long long N,
    float c0, int n, int lo, int s, int periodic,
    unsigned long long* __restrict__ rho, unsigned long long* __restrict__ escaped){
  const float fn = (float)n;
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  unsigned int esc_local = 0;
  // whole warps iterate together (the loop bound is the warp's first
  // particle) so that neighbouring lanes can merge their contributions
  for (long long pw = bi.x * (long long)blockDim.x + (threadIdx.x & ~31); pw < N;
       pw += (long long)bi.gx * blockDim.x) {
    const long long p = pw + lane;
    bool act = p < N;
    int x0 = 0, x1 = 0, y0 = 0, y1 = 0, z0 = 0, z1 = 0, dx = 0, dy = 0, dz = 0;
    if (act) {
      float4 x = pos[p];
      if (DRIFT) {
        float4 v = mom[p];
        x.x = __fadd_rn(x.x, __fmul_rn(v.x, c0));
        x.y = __fadd_rn(x.y, __fmul_rn(v.y, c0));
        x.z = __fadd_rn(x.z, __fmul_rn(v.z, c0));
        if (periodic) {
          if (x.x < 0.f) x.x = __fadd_rn(x.x, fn);
          if (x.x >= fn) x.x = __fsub_rn(x.x, fn);
          if (x.y < 0.f) x.y = __fadd_rn(x.y, fn);
          if (x.y >= fn) x.y = __fsub_rn(x.y, fn);
          if (x.z < 0.f) x.z = __fadd_rn(x.z, fn);
          if (x.z >= fn) x.z = __fsub_rn(x.z, fn);
        }
        pos[p] = x;
      }
      int ix, iy, iz;
      cic_axis(x.x, ix, dx);
      cic_axis(x.y, iy, dy);
      cic_axis(x.z, iz, dz);
      if (periodic) {
        // a wrapped position gives i in [-1, n-1]; anything else (a drift of
        // more than a box length) is counted as escaped, never indexed
        if (ix < -1 || ix > n - 1 || iy < -1 || iy > n - 1 || iz < -1 || iz > n - 1) {
          act = false;
        } else {
          x0 = ix < 0 ? ix + n : ix;  x1 = x0 + 1 == n ? 0 : x0 + 1;
          y0 = iy < 0 ? iy + n : iy;  y1 = y0 + 1 == n ? 0 : y0 + 1;
          z0 = iz < 0 ? iz + n : iz;  z1 = z0 + 1 == n ? 0 : z0 + 1;
        }
      } else {
        const int hi = lo + s - 1;
        if (ix < lo || ix + 1 > hi || iy < lo || iy + 1 > hi || iz < lo || iz + 1 > hi) {
          act = false;
        } else {
          x0 = ix; x1 = ix + 1; y0 = iy; y1 = iy + 1; z0 = iz; z1 = iz + 1;
        }
      }
      if (!act) ++esc_local;
    }
    const unsigned long long wx0 = 65536u - dx, wx1 = dx;
    const unsigned long long wy0 = 65536u - dy, wy1 = dy;
    const unsigned long long wz0 = 65536u - dz, wz1 = dz;
    const unsigned long long a00 = wy0 * wz0, a10 = wy1 * wz0, a01 = wy0 * wz1,
                             a11 = wy1 * wz1;
    // contributions to the x0 column (b) and the x1 column (c) of the cell
    unsigned long long b00 = wx0 * a00, b10 = wx0 * a10, b01 = wx0 * a01, b11 = wx0 * a11;
    unsigned long long c00 = wx1 * a00, c10 = wx1 * a10, c01 = wx1 * a01, c11 = wx1 * a11;
    // 1. lanes in the cell of the lane before them continue its run; each
    // run's eight sums are reduced onto its first lane (the head), which
    // alone issues atomics
    const int pact = __shfl_up_sync(FULL, act ? 1 : 0, 1);
    const int sx0 = __shfl_up_sync(FULL, x0, 1), sy0 = __shfl_up_sync(FULL, y0, 1);
    const int sz0 = __shfl_up_sync(FULL, z0, 1);
    const bool same = lane > 0 && act && pact != 0 && sx0 == x0 && sy0 == y0 && sz0 == z0;
    const unsigned cont = __ballot_sync(FULL, same);
    if (cont) {
      // last lane of my run: the one before the next lane that does not continue
      const unsigned brk = ~cont & (0xfffffffeu << lane);
      const int rend = brk ? __ffs(brk) - 2 : 31;
      for (int o = 1; o < 32; o <<= 1) {
        const bool in = lane + o <= rend;
        if (!__any_sync(FULL, in)) break;
#define PM_RUN_ADD(v) { const unsigned long long t_ = __shfl_down_sync(FULL, v, o); if (in) v += t_; }
        PM_RUN_ADD(b00) PM_RUN_ADD(b10) PM_RUN_ADD(b01) PM_RUN_ADD(b11)
        PM_RUN_ADD(c00) PM_RUN_ADD(c10) PM_RUN_ADD(c01) PM_RUN_ADD(c11)
#undef PM_RUN_ADD
      }
    }
    // 2. the x1 column of a head is the x0 column of the next head when their
    // cells are x-neighbours: the next head adds it to its own atomics
    const bool head = act && !same;
    const unsigned heads = __ballot_sync(FULL, head);
    const unsigned below = heads & ((1u << lane) - 1u);
    const int ph = below ? 31 - __clz(below) : lane;
    const int px1 = __shfl_sync(FULL, x1, ph), py0 = __shfl_sync(FULL, y0, ph);
    const int pz0 = __shfl_sync(FULL, z0, ph);
    const unsigned long long q00 = __shfl_sync(FULL, c00, ph), q10 = __shfl_sync(FULL, c10, ph);
    const unsigned long long q01 = __shfl_sync(FULL, c01, ph), q11 = __shfl_sync(FULL, c11, ph);
    const bool take = head && below != 0u && px1 == x0 && py0 == y0 && pz0 == z0;
    const unsigned takes = __ballot_sync(FULL, take);
    const unsigned above = heads & (0xfffffffeu << lane);
    const bool given = above != 0u && ((takes >> (__ffs(above) - 1)) & 1u);
    if (head) {
      const long long r00 = ((long long)z0 * n + y0) * n, r10 = ((long long)z0 * n + y1) * n;
      const long long r01 = ((long long)z1 * n + y0) * n, r11 = ((long long)z1 * n + y1) * n;
      atomicAdd(rho + r00 + x0, b00 + (take ? q00 : 0ull));
      atomicAdd(rho + r10 + x0, b10 + (take ? q10 : 0ull));
      atomicAdd(rho + r01 + x0, b01 + (take ? q01 : 0ull));
      atomicAdd(rho + r11 + x0, b11 + (take ? q11 : 0ull));
      if (!given) {
        atomicAdd(rho + r00 + x1, c00);
        atomicAdd(rho + r10 + x1, c10);
        atomicAdd(rho + r01 + x1, c01);
        atomicAdd(rho + r11 + x1, c11);
      }
    }
  }
  {
    unsigned int w = esc_local;
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    if ((threadIdx.x & 31) == 0 && w) atomicAdd(escaped, (unsigned long long)w);
  }
}

template <bool DRIFT>
__global__ void __launch_bounds__(256) k_drift_deposit(
    float4* __restrict__ pos, const float4* __restrict__ mom, long long N,
    float c0, int n, int lo, int s, int periodic,
    unsigned long long* __restrict__ rho, unsigned long long* __restrict__ escaped) {
  pdl_wait();
  pdl_release();
  d_drift_deposit<DRIFT>(bi_native(), pos, mom, N, c0, n, lo, s, periodic, rho, escaped);
}

void launch_drift_deposit(cudaStream_t st, int grid, float4* pos, const float4* mom,
                          long long N, float c0, bool drift, int n, int lo, int s,
                          int periodic, unsigned long long* rho,
                          unsigned long long* escaped) {
  if (N <= 0) return;
  if (drift)
    launch_pdl(k_drift_deposit<true>, dim3(grid), dim3(256), 0, st, pos, mom, N, c0, n, lo, s,
               periodic, rho, escaped);
  else
    launch_pdl(k_drift_deposit<false>, dim3(grid), dim3(256), 0, st, pos, mom, N, c0, n, lo, s,
               periodic, rho, escaped);
  note_launch();
}

// ---------------------------------------------------------------------------
// Mean-density term of a spherical keep region (Table 1's domain): the CIC
// image of the ball |x - c| <= R on every cell of the (even-sided, centred)
// cube, written to the full-mesh array W [z][y][x], and its moments (sum W, sum W y_a,
// sum W y_a y_b, y the cell centre - c) reduced in a fixed order into
// out[0..9] (the layout of the source kernel's background moments).  Per
// cell: 1 when |y| + sqrt(3) <= R, 0 when |y| - sqrt(3) >= R, otherwise the
// z integral of the tent over the ball's chord in closed form,
// T(h - y_z) - T(-h - y_z) with h = sqrt(R^2 - X^2 - Y^2), summed over the
// four quadrants of the x-y tent support with the product Gauss-Legendre
// rule `rule` (nodes xi on [0, 1], weights times the tent 1 - xi).  FP32.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float tent_cdf(float u) {
  if (u <= -1.0f) return 0.0f;
  if (u <= 0.0f) return 0.5f * (u + 1.0f) * (u + 1.0f);
  if (u <= 1.0f) return 1.0f - 0.5f * (1.0f - u) * (1.0f - u);
  return 1.0f;
}

__global__ void __launch_bounds__(256) k_ball_w(float* __restrict__ W, int n, int lo, int s,
                                                double R, BallRule rule,
                                                double* __restrict__ partial,
                                                unsigned int* counter, double* __restrict__ out) {
  // The cube is centred on c and W is even in each coordinate, so one warp
  // takes an x row of the octant i, j, k >= s/2 and writes each value to
  // its eight mirror cells; a cell on the ball's surface is integrated by
  // the whole warp (the 4 G^2 rule points split over the lanes).
  constexpr unsigned FULL = 0xffffffffu;
  constexpr int NQ = 4 * BALL_GL * BALL_GL;
  double m[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  const int half = s / 2, lane = threadIdx.x & 31;
  const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  const float R2 = (float)(R * R);
  const double c = 0.5 * n;
  for (int row = gw; row < half * half; row += nw) {
    const int jj = half + row % half, kk = half + row / half;
    for (int x0 = half; x0 < s; x0 += 32) {
      const int ii = x0 + lane;
      const bool valid = ii < s;
      const double yx = lo + ii + 0.5 - c, yy = lo + jj + 0.5 - c, yz = lo + kk + 0.5 - c;
      const double r = sqrt(yx * yx + yy * yy + yz * yz);
      const int cls = !valid ? -1
                      : (r + 1.7320508075688772 <= R ? 1
                                                      : (r - 1.7320508075688772 >= R ? 0 : 2));
      float w = cls == 1 ? 1.0f : 0.0f;
      unsigned shell = __ballot_sync(FULL, cls == 2);
      while (shell) {
        const int src = __ffs(shell) - 1;
        shell &= shell - 1;
        const float ax = __shfl_sync(FULL, (float)yx, src);
        const float ay = __shfl_sync(FULL, (float)yy, src);
        const float az = __shfl_sync(FULL, (float)yz, src);
        float part = 0.0f;
        for (int e = lane; e < NQ; e += 32) {
          const int q = e / (BALL_GL * BALL_GL), g = (e / BALL_GL) % BALL_GL,
                    h = e % BALL_GL;
          const float X = ax + ((q & 1) ? rule.xi[g] : -rule.xi[g]);
          const float Y = ay + ((q & 2) ? rule.xi[h] : -rule.xi[h]);
          const float h2 = R2 - X * X - Y * Y;
          if (h2 > 0.0f) {
            const float hz = sqrtf(h2);
            part += rule.om[g] * rule.om[h] * (tent_cdf(hz - az) - tent_cdf(-hz - az));
          }
        }
        part = warp_sumf_all(part);
        if (lane == src) w = part;
      }
      if (!valid) continue;
      const double wd = (double)w;
#pragma unroll
      for (int mirror = 0; mirror < 8; ++mirror) {
        const int i2 = (mirror & 1) ? s - 1 - ii : ii;
        const int j2 = (mirror & 2) ? s - 1 - jj : jj;
        const int k2 = (mirror & 4) ? s - 1 - kk : kk;
        W[((long long)(lo + k2) * n + (lo + j2)) * n + (lo + i2)] = w;
        const double px = (mirror & 1) ? -yx : yx, py = (mirror & 2) ? -yy : yy,
                     pz = (mirror & 4) ? -yz : yz;
        m[0] += wd;
        m[1] += wd * px;
        m[2] += wd * py;
        m[3] += wd * pz;
        m[4] += wd * px * px;
        m[5] += wd * py * py;
        m[6] += wd * pz * pz;
        m[7] += wd * px * py;
        m[8] += wd * px * pz;
        m[9] += wd * py * pz;
      }
    }
  }
  // block sums (fixed order), then the last block folds the partials in order
  __shared__ double sm[8][10];
  const int warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < 10; ++q) {
    const double v = warp_sum(m[q]);
    if (lane == 0) sm[warp][q] = v;
  }
  __syncthreads();
  __shared__ bool last;
  if (threadIdx.x == 0) {
    for (int q = 0; q < 10; ++q) {
      double v = 0.0;
      for (int w8 = 0; w8 < (int)(blockDim.x >> 5); ++w8) v += sm[w8][q];
      partial[blockIdx.x * 10 + q] = v;
    }
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  if (threadIdx.x < 10) {
    double v = 0.0;
    for (unsigned b = 0; b < gridDim.x; ++b) v += __ldcg(partial + b * 10 + threadIdx.x);
    out[threadIdx.x] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) *counter = 0u;
}

void launch_ball_w(cudaStream_t st, float* W, int n, int lo, int s, double R,
                   const BallRule& rule, double* partial, unsigned int* counter, double* out) {
  // one warp per octant row (the cube side is even), 8 warps per block
  const long long rows = (long long)(s / 2) * (s / 2);
  const int g = (int)std::max<long long>(1, std::min<long long>((rows + 7) / 8, 1216));
  k_ball_w<<<g, 256, 0, st>>>(W, n, lo, s, R, rule, partial, counter, out);
  note_launch();
}

// ---------------------------------------------------------------------------
// TSC variant of the drift + deposit (Sec. 2.4 footnote: CIC or TSC).  Per
// axis the particle's cell i = floor(u) and its position in the cell in
// Q16, q = floor(2^16 u) - 2^16 i, give the weights of nodes i-1, i, i+1:
// (2^16 - q)^2 >> 17, the rest, q^2 >> 17 (the kernel (1/2 -+ d)^2 / 2 and
// 3/4 - d^2 at d = u - i - 1/2), summing to exactly 2^16; the 27 products
// (<= 2^48, 2^48 in total) go to int64 cell counts.  Periodic: nodes wrap;
// open: a particle with a node outside the cube deposits nothing (escaped).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void tsc_axis(float u, int& i, unsigned int w[3]) {
  const int iq = __float2int_rd(__fmul_rn(u, 65536.0f));
  i = iq >> 16;
  const unsigned long long q = (unsigned long long)(iq & 0xffff);
  const unsigned long long a = 65536ull - q;
  w[0] = (unsigned int)((a * a) >> 17);
  w[2] = (unsigned int)((q * q) >> 17);
  w[1] = 65536u - w[0] - w[2];
}

template <bool DRIFT>
__global__ void __launch_bounds__(256) k_drift_deposit_tsc(
    float4* __restrict__ pos, const float4* __restrict__ mom, long long N, float c0, int n,
    int lo, int s, int periodic, unsigned long long* __restrict__ rho,
    unsigned long long* __restrict__ escaped) {
  const float fn = (float)n;
  unsigned int esc_local = 0;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N;
       p += (long long)gridDim.x * blockDim.x) {
    float4 x = pos[p];
    if (DRIFT) {
      const float4 v = mom[p];
      x.x = __fadd_rn(x.x, __fmul_rn(v.x, c0));
      x.y = __fadd_rn(x.y, __fmul_rn(v.y, c0));
      x.z = __fadd_rn(x.z, __fmul_rn(v.z, c0));
      if (periodic) {
        if (x.x < 0.f) x.x = __fadd_rn(x.x, fn);
        if (x.x >= fn) x.x = __fsub_rn(x.x, fn);
        if (x.y < 0.f) x.y = __fadd_rn(x.y, fn);
        if (x.y >= fn) x.y = __fsub_rn(x.y, fn);
        if (x.z < 0.f) x.z = __fadd_rn(x.z, fn);
        if (x.z >= fn) x.z = __fsub_rn(x.z, fn);
      }
      pos[p] = x;
    }
    int i3[3];
    unsigned int w[3][3];
    tsc_axis(x.x, i3[0], w[0]);
    tsc_axis(x.y, i3[1], w[1]);
    tsc_axis(x.z, i3[2], w[2]);
    bool ok = true;
    int nd[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (periodic) {
        ok = ok && i3[a] >= 0 && i3[a] <= n - 1;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const int v = i3[a] - 1 + c;
          nd[a][c] = v < 0 ? v + n : (v >= n ? v - n : v);
        }
      } else {
        ok = ok && i3[a] - 1 >= lo && i3[a] + 1 <= lo + s - 1;
#pragma unroll
        for (int c = 0; c < 3; ++c) nd[a][c] = i3[a] - 1 + c;
      }
    }
    if (!ok) {
      ++esc_local;
      continue;
    }
#pragma unroll
    for (int cz = 0; cz < 3; ++cz)
#pragma unroll
      for (int cy = 0; cy < 3; ++cy) {
        const unsigned long long wyz = (unsigned long long)w[1][cy] * w[2][cz];
        const long long row = ((long long)nd[2][cz] * n + nd[1][cy]) * n;
#pragma unroll
        for (int cx = 0; cx < 3; ++cx) atomicAdd(rho + row + nd[0][cx], wyz * w[0][cx]);
      }
  }
  unsigned int w = esc_local;
  for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
  if ((threadIdx.x & 31) == 0 && w) atomicAdd(escaped, (unsigned long long)w);
}

void launch_drift_deposit_tsc(cudaStream_t st, long long N, float4* pos, const float4* mom,
                              float c0, bool drift, int n, int lo, int s, int periodic,
                              unsigned long long* rho, unsigned long long* escaped) {
  if (N <= 0) return;
  const int g = (int)std::min<long long>((N + 255) / 256, 152 * 16);
  if (drift)
    k_drift_deposit_tsc<true><<<g, 256, 0, st>>>(pos, mom, N, c0, n, lo, s, periodic, rho,
                                                 escaped);
  else
    k_drift_deposit_tsc<false><<<g, 256, 0, st>>>(pos, mom, N, c0, n, lo, s, periodic, rho,
                                                  escaped);
  note_launch();
}

// ---------------------------------------------------------------------------
// Deterministic "last block finishes" reduction helpers.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool arrive_last(unsigned int* counter) {
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned int t = atomicAdd(counter, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  return last;
}

__device__ __forceinline__ double i128_to_double(__int128 v) {
  bool neg = v < 0;
  unsigned __int128 u = neg ? (unsigned __int128)(-v) : (unsigned __int128)v;
  double d = (double)(unsigned long long)(u >> 64) * 18446744073709551616.0 +
             (double)(unsigned long long)u;
  return neg ? -d : d;
}

__device__ __forceinline__ __int128 shfl_xor_i128(__int128 v, int o) {
  unsigned long long lo = (unsigned long long)v;
  long long hi = (long long)(v >> 64);
  lo = __shfl_xor_sync(0xffffffffu, lo, o);
  hi = __shfl_xor_sync(0xffffffffu, hi, o);
  return ((__int128)hi << 64) | (__int128)lo;
}

// ---------------------------------------------------------------------------
// K2: source on the active cube from the int64 counts.
//   delta = rho / (2^48 nbar) - [cell centre inside the keep cube]
//   f     = S delta                          (double-float, hi/lo planes)
// clears rho for the next deposit, flags counts > 2^62, accumulates ||f||^2
// and, in the open phase, the exact integer moments
//   sum rho, sum rho X_a, sum rho X_a X_b   with X = 2 (cell centre - c),
// finished by the last block into moments of delta (q0, d_a, S_ab) in cell
// units.  out[0] = ||f||^2, out[1..10] = moments.
// ---------------------------------------------------------------------------
constexpr int SRC_NV = 10;

template <bool MOMENTS>
__device__ __forceinline__ void d_source(const BI& bi, 
    unsigned long long* __restrict__ rho, int n, int lo, int s, Grid fh, Grid fl,
    df invM, df S, const df* __restrict__ bgw, const float* __restrict__ ballw,
    double* __restrict__ partial_f2,
    __int128* __restrict__ partial_m, unsigned int* counter, double* __restrict__ out,
    const double* __restrict__ bgm, double invM2_hi, int* __restrict__ overflow){
  __int128 acc[SRC_NV];
#pragma unroll
  for (int q = 0; q < SRC_NV; ++q) acc[q] = 0;
  // moments of the thread's column: sum c, c Z, c Z^2 with the count split
  // c = c1 2^32 + c0 so that every partial sum is exact in int64 (at most
  // 64 cells of |Z| < 2^11 per thread); the X, Y factors are constant along
  // the column and applied once at the end in int128
  long long m0[2] = {0, 0}, mz[2] = {0, 0}, mzz[2] = {0, 0};
  float f2 = 0.f;
  // block (32, 8) covers an x-y tile; the grid's z dimension strides over
  // planes, ZU planes per round with all loads issued before any use
  constexpr int ZU = 4;
  const int i = bi.x * blockDim.x + threadIdx.x;
  const int j = bi.y * blockDim.y + threadIdx.y;
  const bool in_xy = i < s && j < s;
  const int gi = lo + i, gj = lo + j;
  // mean-density weight W = w_x w_y w_z (per-axis CIC image of the keep
  // interval, indexed by global cell; all ones in the periodic phase)
  df wxy{0.0f, 0.0f};
  if (in_xy) wxy = df_mul(bgw[gi], bgw[gj]);
  for (int k0 = bi.z; k0 < s && in_xy; k0 += ZU * bi.gz) {
    unsigned long long cnts[ZU];
#pragma unroll
    for (int u = 0; u < ZU; ++u) {
      int k = k0 + u * bi.gz;
      cnts[u] = k < s ? rho[((long long)(lo + k) * n + gj) * n + gi] : 0ull;
    }
#pragma unroll
    for (int u = 0; u < ZU; ++u) {
    int k = k0 + u * bi.gz;
    if (k >= s) break;
    int gk = lo + k;
    unsigned long long cnt = cnts[u];
    rho[((long long)gk * n + gj) * n + gi] = 0ull;
    if (cnt > (1ull << 62)) atomicOr(overflow, 1);
    long long c = (long long)cnt;
    df d = df_mul(df_from_u64(cnt), invM);
    // ballw (spherical keep region): the mean density's image per cell
    const df w = ballw ? df{ballw[((long long)gk * n + gj) * n + gi], 0.0f}
                       : df_mul(wxy, bgw[gk]);
    d = df_add(d, df{-w.hi, -w.lo});
    df f = df_mul(d, S);
    int fi = gidx(fh, i, j, k);
    fh.base[fi] = f.hi;
    fl.base[fi] = f.lo;
    f2 = __fmaf_rn(f.hi, f.hi, f2);
    if (MOMENTS) {
      const int Z = 2 * gk + 1 - n;
      const long long c0 = (long long)(cnt & 0xffffffffull), c1 = (long long)(cnt >> 32);
      m0[0] += c0;
      m0[1] += c1;
      mz[0] += c0 * Z;
      mz[1] += c1 * Z;
      mzz[0] += c0 * (long long)(Z * Z);
      mzz[1] += c1 * (long long)(Z * Z);
    }
    }
  }
  if (MOMENTS && in_xy) {
    const long long X = 2 * gi + 1 - n, Y = 2 * gj + 1 - n;
    const __int128 M0 = (__int128)m0[0] + ((__int128)m0[1] << 32);
    const __int128 MZ = (__int128)mz[0] + ((__int128)mz[1] << 32);
    const __int128 MZZ = (__int128)mzz[0] + ((__int128)mzz[1] << 32);
    acc[0] = M0;
    acc[1] = M0 * X;
    acc[2] = M0 * Y;
    acc[3] = MZ;
    acc[4] = M0 * (X * X);
    acc[5] = M0 * (Y * Y);
    acc[6] = MZZ;
    acc[7] = M0 * (X * Y);
    acc[8] = MZ * X;
    acc[9] = MZ * Y;
  }
  // block reduction: ||f||^2 in double, moments in int128
  __shared__ double sf[32];
  __shared__ __int128 sm[32 * SRC_NV];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const unsigned bid = bi.x + bi.gx * (bi.y + bi.gy * bi.z);
  const unsigned nblk = bi.gx * bi.gy * bi.gz;
  int lane = tid & 31, warp = tid >> 5, nw = (blockDim.x * blockDim.y) >> 5;
  float wf = warp_sumf_all(f2);
  if (lane == 0) sf[warp] = (double)wf;
  if (MOMENTS) {
#pragma unroll
    for (int q = 0; q < SRC_NV; ++q) {
      __int128 v = acc[q];
      for (int o = 16; o > 0; o >>= 1) v += shfl_xor_i128(v, o);
      if (lane == 0) sm[warp * SRC_NV + q] = v;
    }
  }
  __syncthreads();
  __shared__ bool last;
  if (tid == 0) {
    double tf = 0.0;
    for (int q = 0; q < nw; ++q) tf += sf[q];
    partial_f2[bid] = tf;
    if (MOMENTS) {
      for (int q = 0; q < SRC_NV; ++q) {
        __int128 v = 0;
        for (int u = 0; u < nw; ++u) v += sm[u * SRC_NV + q];
        partial_m[bid * SRC_NV + q] = v;
      }
    }
    __threadfence();
    last = (atomicAdd(counter, 1u) == nblk - 1);
  }
  __syncthreads();
  if (!last) return;
  // the last block folds all partials: strided per thread, then block-wide
  double tf = 0.0;
  __int128 tot[SRC_NV];
#pragma unroll
  for (int q = 0; q < SRC_NV; ++q) tot[q] = 0;
  const int nth = blockDim.x * blockDim.y;
  for (unsigned b = tid; b < nblk; b += nth) {
    tf += __ldcg(partial_f2 + b);
    if (MOMENTS) {
#pragma unroll
      for (int q = 0; q < SRC_NV; ++q) {
        const unsigned long long* pp =
            reinterpret_cast<const unsigned long long*>(partial_m + b * SRC_NV + q);
        unsigned long long plo = __ldcg(pp), phi = __ldcg(pp + 1);
        tot[q] += (__int128)(((unsigned __int128)phi << 64) | plo);
      }
    }
  }
  tf = warp_sum(tf);
  if (MOMENTS) {
#pragma unroll
    for (int q = 0; q < SRC_NV; ++q)
      for (int o = 16; o > 0; o >>= 1) tot[q] += shfl_xor_i128(tot[q], o);
  }
  __syncthreads();
  if (lane == 0) {
    sf[warp] = tf;
    if (MOMENTS)
      for (int q = 0; q < SRC_NV; ++q) sm[warp * SRC_NV + q] = tot[q];
  }
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += sf[w];
    out[0] = t;
    if (MOMENTS) {
      __int128 T[SRC_NV];
      for (int q = 0; q < SRC_NV; ++q) {
        T[q] = 0;
        for (int w = 0; w < nw; ++w) T[q] += sm[w * SRC_NV + q];
      }
      // moments of rho / M in cell units (X = 2y) minus the background's
      double m[SRC_NV];
      m[0] = i128_to_double(T[0]) * invM2_hi;
      for (int q = 1; q < 4; ++q) m[q] = i128_to_double(T[q]) * invM2_hi * 0.5;
      for (int q = 4; q < 10; ++q) m[q] = i128_to_double(T[q]) * invM2_hi * 0.25;
      for (int q = 0; q < SRC_NV; ++q) out[1 + q] = m[q] - bgm[q];
    }
    *counter = 0u;
  }
}

template <bool MOMENTS>
__global__ void __launch_bounds__(256) k_source(
    unsigned long long* __restrict__ rho, int n, int lo, int s, Grid fh, Grid fl,
    df invM, df S, const df* __restrict__ bgw, const float* __restrict__ ballw,
    double* __restrict__ partial_f2,
    __int128* __restrict__ partial_m, unsigned int* counter, double* __restrict__ out,
    const double* __restrict__ bgm, double invM2_hi, int* __restrict__ overflow) {
  pdl_wait();
  pdl_release();
  d_source<MOMENTS>(bi_native(), rho, n, lo, s, fh, fl, invM, S, bgw, ballw, partial_f2,
                    partial_m, counter, out, bgm, invM2_hi, overflow);
}

dim3 source_grid(int s) {
  return dim3((unsigned)((s + 31) / 32), (unsigned)((s + 7) / 8), (unsigned)(s < 16 ? s : 16));
}

void launch_source(cudaStream_t st, int grid, unsigned long long* rho, int n, int lo,
                   int s, Grid fh, Grid fl, double invM, double S, const df* bgw,
                   const float* ballw,
                   bool moments, double* partial_f2, void* partial_m,
                   unsigned int* counter, double* out, const double* bgm, int* overflow) {
  df invMd, Sd;
  invMd.hi = (float)invM;
  invMd.lo = (float)(invM - (double)invMd.hi);
  Sd.hi = (float)S;
  Sd.lo = (float)(S - (double)Sd.hi);
  if (moments)
    launch_pdl(k_source<true>, source_grid(s), dim3(32, 8), 0, st, rho, n, lo, s, fh, fl, invMd,
               Sd, bgw, ballw, partial_f2, (__int128*)partial_m, counter, out, bgm, invM,
               overflow);
  else
    launch_pdl(k_source<false>, source_grid(s), dim3(32, 8), 0, st, rho, n, lo, s, fh, fl, invMd,
               Sd, bgw, ballw, partial_f2, (__int128*)partial_m, counter, out, bgm, invM,
               overflow);
  note_launch();
}

// ---------------------------------------------------------------------------
// Source from a caller's FP64 delta on the whole n^3 mesh (pm_potential):
// f = S delta split into hi/lo, ||f||^2, and FP64 moments of delta.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_source_f64(
    const double* __restrict__ delta, int n, Grid fh, Grid fl, double S, int moments,
    double* __restrict__ partial, unsigned int* counter, double* __restrict__ out) {
  double acc[11];
#pragma unroll
  for (int q = 0; q < 11; ++q) acc[q] = 0.0;
  const long long total = (long long)n * n * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int i = (int)(t % n);
    long long r = t / n;
    int j = (int)(r % n);
    int k = (int)(r / n);
    double d = delta[t];
    double f = S * d;
    float hi = (float)f;
    float lo = (float)(f - (double)hi);
    int fi = gidx(fh, i, j, k);
    fh.base[fi] = hi;
    fl.base[fi] = lo;
    acc[0] += f * f;
    if (moments) {
      double x = i + 0.5 - 0.5 * n, y = j + 0.5 - 0.5 * n, z = k + 0.5 - 0.5 * n;
      acc[1] += d;
      acc[2] += d * x;
      acc[3] += d * y;
      acc[4] += d * z;
      acc[5] += d * x * x;
      acc[6] += d * y * y;
      acc[7] += d * z * z;
      acc[8] += d * x * y;
      acc[9] += d * x * z;
      acc[10] += d * y * z;
    }
  }
  __shared__ double sm[32 * 11];
  block_sum<11>(acc, sm);
  if (threadIdx.x == 0)
    for (int q = 0; q < 11; ++q) partial[blockIdx.x * 11 + q] = acc[q];
  if (!arrive_last(counter)) return;
  if (threadIdx.x == 0) {
    for (int q = 0; q < 11; ++q) {
      double v = 0.0;
      for (unsigned b = 0; b < gridDim.x; ++b) v += __ldcg(partial + b * 11 + q);
      out[q] = v;
    }
    *counter = 0u;
  }
}

void launch_source_f64(cudaStream_t st, int grid, const double* delta, int n, Grid fh,
                       Grid fl, double S, bool moments, double* partial,
                       unsigned int* counter, double* out) {
  k_source_f64<<<grid, 256, 0, st>>>(delta, n, fh, fl, S, moments ? 1 : 0, partial,
                                     counter, out);
  note_launch();
}

// ---------------------------------------------------------------------------
// Right-hand side of an implicit diffusion substep (backward Euler on Eq. 4):
// g = scale * src - sig * Phi_old in double-float on the cube interior,
// written to (gh, gl); with `stash` the source is first copied to (qh, ql).
// ||g||^2 into out[0] (deterministic block partials).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_diff_rhs(Grid sh, Grid sl, float scale_hi,
                                                  float scale_lo, Grid ph, Grid pl, float sig_hi,
                                                  float sig_lo,
                                                  Grid gh, Grid gl, Grid qh, Grid ql, int stash,
                                                  double* __restrict__ partial,
                                                  unsigned int* counter,
                                                  double* __restrict__ out) {
  const int s = ph.s;
  const long long total = (long long)s * s * s;
  double acc[1] = {0.0};
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % s);
    const long long r = t / s;
    const int j = (int)(r % s), k = (int)(r / s);
    const int cs = gidx(sh, i, j, k), cp = gidx(ph, i, j, k), cg = gidx(gh, i, j, k);
    const df src{sh.base[cs], sl.base[cs]};
    if (stash) {
      const int cq = gidx(qh, i, j, k);
      qh.base[cq] = src.hi;
      ql.base[cq] = src.lo;
    }
    const df a = df_mul(src, df{scale_hi, scale_lo});
    const df b = df_mul(df{ph.base[cp], pl.base[cp]}, df{-sig_hi, -sig_lo});
    const df g = df_add(a, b);
    gh.base[cg] = g.hi;
    gl.base[cg] = g.lo;
    acc[0] += (double)g.hi * (double)g.hi;
  }
  __shared__ double sm[32];
  block_sum<1>(acc, sm);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc[0];
  if (!arrive_last(counter)) return;
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (unsigned b = 0; b < gridDim.x; ++b) v += __ldcg(partial + b);
    out[0] = v;
    *counter = 0u;
  }
}

void launch_diff_rhs(cudaStream_t st, int grid, Grid sh, Grid sl, double scale, Grid ph,
                     Grid pl, double sig, Grid gh, Grid gl, Grid qh, Grid ql, bool stash,
                     double* partial, unsigned int* counter, double* out) {
  const float shi = (float)scale, slo = (float)(scale - (double)shi);
  const float ghi = (float)sig, glo = (float)(sig - (double)ghi);
  k_diff_rhs<<<grid, 256, 0, st>>>(sh, sl, shi, slo, ph, pl, ghi, glo, gh, gl, qh, ql,
                                   stash ? 1 : 0, partial, counter, out);
  note_launch();
}

// ---------------------------------------------------------------------------
// K3: open-boundary ghost layer.  At each ghost-cell centre r (relative to
// the box centre): Phi = -(S/4pi) [q0/r + d.r/r^3 + r.Q.r/(2 r^5)],
// Q_ab = 3 S_ab - delta_ab tr(S).  mom = (q0, dx, dy, dz, Sxx, Syy, Szz, Sxy,
// Sxz, Syz).  Written to the hi/lo planes (lo = 0 when want_lo == 0).
// ---------------------------------------------------------------------------
// ghost cell t of the 6 (s+2)^2 faces of a cube of side s: its (i, j, k)
// in cube coordinates (-1 or s on the face's axis)
__device__ __forceinline__ bool ghost_cell(long long t, int s, int& i, int& j, int& k) {
  const int P = s + 2;
  const long long per_face = (long long)P * P;
  if (t >= 6 * per_face) return false;
  int face = (int)(t / per_face);
  int rem = (int)(t % per_face);
  int u = rem % P - 1, v = rem / P - 1;
  int side = (face & 1) ? s : -1;
  switch (face >> 1) {
    case 0: i = side; j = u; k = v; break;
    case 1: j = side; i = u; k = v; break;
    default: k = side; i = u; j = v; break;
  }
  return true;
}

// the multipole potential at the centre of cube cell (i, j, k) of a cube at
// lo in an n^3 mesh
__device__ __forceinline__ double ghost_value(int n, int lo, int i, int j, int k,
                                              const double* __restrict__ mom, double S) {
  const double q0 = mom[0], dx = mom[1], dy = mom[2], dz = mom[3];
  const double sxx = mom[4], syy = mom[5], szz = mom[6];
  const double sxy = mom[7], sxz = mom[8], syz = mom[9];
  const double tr = sxx + syy + szz;
  const double qxx = 3 * sxx - tr, qyy = 3 * syy - tr, qzz = 3 * szz - tr;
  const double qxy = 3 * sxy, qxz = 3 * sxz, qyz = 3 * syz;
  double x = lo + i + 0.5 - 0.5 * n, y = lo + j + 0.5 - 0.5 * n, z = lo + k + 0.5 - 0.5 * n;
  double r2 = x * x + y * y + z * z;
  double qr = qxx * x * x + qyy * y * y + qzz * z * z +
              2.0 * (qxy * x * y + qxz * x * z + qyz * y * z);
  // q0/r + d.x/r^3 + qr/(2 r^5) from one reciprocal square root: the float
  // estimate refined by two Newton steps in FP64, ri <- ri (3 - r2 ri^2) / 2,
  // each squaring the relative error (1e-7 -> 1e-14 -> double rounding);
  // FP64 divisions and square roots are long sequences on this part
  double ri = (double)rsqrtf((float)r2);
  ri = ri * (1.5 - 0.5 * r2 * ri * ri);
  ri = ri * (1.5 - 0.5 * r2 * ri * ri);
  const double ri2 = ri * ri;
  return -(S / (4.0 * 3.14159265358979323846)) * ri *
         (q0 + ri2 * ((dx * x + dy * y + dz * z) + 0.5 * qr * ri2));
}

// The same multipole value in FP32 throughout
__device__ __forceinline__ float ghost_value_f(int n, int lo, int i, int j, int k,
                                               const double* __restrict__ mom, float S) {
  const float q0 = (float)mom[0], dx = (float)mom[1], dy = (float)mom[2], dz = (float)mom[3];
  const float sxx = (float)mom[4], syy = (float)mom[5], szz = (float)mom[6];
  const float sxy = (float)mom[7], sxz = (float)mom[8], syz = (float)mom[9];
  const float tr = sxx + syy + szz;
  const float qxx = 3.0f * sxx - tr, qyy = 3.0f * syy - tr, qzz = 3.0f * szz - tr;
  const float qxy = 3.0f * sxy, qxz = 3.0f * sxz, qyz = 3.0f * syz;
  const float h = 0.5f * (float)n;
  const float x = (float)(lo + i) + 0.5f - h, y = (float)(lo + j) + 0.5f - h;
  const float z = (float)(lo + k) + 0.5f - h;
  const float r2 = x * x + y * y + z * z;
  const float qr = qxx * x * x + qyy * y * y + qzz * z * z +
                   2.0f * (qxy * x * y + qxz * x * z + qyz * y * z);
  const float ri = rsqrtf(r2), ri2 = ri * ri;
  return -(S / (4.0f * 3.14159265f)) * ri *
         (q0 + ri2 * ((dx * x + dy * y + dz * z) + 0.5f * qr * ri2));
}

// the values into (ph, pl) and, when ph2.base is not NULL, the same into
// (ph2, pl2) (the second buffer of the defect correction's potential)
__device__ __forceinline__ void d_boundary(const BI& bi, Grid ph, Grid pl, int n, int lo,
                                                  const double* __restrict__ mom,
                                                  double S, int want_lo, Grid ph2, Grid pl2){
  int i, j, k;
  if (!ghost_cell(bi.x * (long long)blockDim.x + threadIdx.x, ph.s, i, j, k)) return;
  const double phi = ghost_value(n, lo, i, j, k, mom, S);
  const float hi = (float)phi;
  const float lov = want_lo ? (float)(phi - (double)hi) : 0.0f;
  int gi = gidx(ph, i, j, k);
  ph.base[gi] = hi;
  pl.base[gi] = lov;
  if (ph2.base) {
    gi = gidx(ph2, i, j, k);
    ph2.base[gi] = hi;
    pl2.base[gi] = lov;
  }
}

__global__ void __launch_bounds__(256) k_boundary(Grid ph, Grid pl, int n, int lo,
                                                  const double* __restrict__ mom,
                                                  double S, int want_lo, Grid ph2, Grid pl2) {
  d_boundary(bi_native(), ph, pl, n, lo, mom, S, want_lo, ph2, pl2);
}

void launch_boundary(cudaStream_t st, Grid ph, Grid pl, int n, int lo, const double* mom,
                     double S, bool want_lo, const Grid* ph2, const Grid* pl2) {
  long long tot = 6LL * (ph.s + 2) * (ph.s + 2);
  int grid = (int)((tot + 255) / 256);
  Grid none{};
  k_boundary<<<grid, 256, 0, st>>>(ph, pl, n, lo, mom, S, want_lo ? 1 : 0,
                                   ph2 ? *ph2 : none, pl2 ? *pl2 : none);
  note_launch();
}

// The ball solve's boundary values: every cell of the padded cube outside
// the mask (ph's mask fields) takes the multipole value, in (ph, pl) and
// (ph2, pl2): the cells next to the mask are its Dirichlet ghosts, the rest
// give the force of particles beyond the mask in the step before they leave.
__global__ void __launch_bounds__(256) k_ball_ghosts(Grid ph, Grid pl, Grid ph2, Grid pl2,
                                                     int n, int lo,
                                                     const double* __restrict__ mom,
                                                     double S) {
  const int s = ph.s, P = s + 2;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)P * P * P) return;
  const int i = (int)(t % P) - 1, j = (int)((t / P) % P) - 1, k = (int)(t / ((long long)P * P)) - 1;
  auto in = [&](int a, int b, int c) {
    return a >= 0 && b >= 0 && c >= 0 && a < s && b < s && c < s && g_in(ph, a, b, c);
  };
  if (in(i, j, k)) return;
  // the Dirichlet ghosts (next to the mask) in FP64 as a hi + lo pair; the
  // cells beyond, read only by the gather of particles beyond the mask, in
  // FP32 (FP64 arithmetic is slow on this part)
  const bool ghost = in(i - 1, j, k) || in(i + 1, j, k) || in(i, j - 1, k) ||
                     in(i, j + 1, k) || in(i, j, k - 1) || in(i, j, k + 1);
  float hi, lov;
  if (ghost) {
    const double phi = ghost_value(n, lo, i, j, k, mom, S);
    hi = (float)phi;
    lov = (float)(phi - (double)hi);
  } else {
    hi = ghost_value_f(n, lo, i, j, k, mom, (float)S);
    lov = 0.0f;
  }
  ph.base[gidx(ph, i, j, k)] = hi;
  pl.base[gidx(pl, i, j, k)] = lov;
  ph2.base[gidx(ph2, i, j, k)] = hi;
  pl2.base[gidx(pl2, i, j, k)] = lov;
}

void launch_ball_ghosts(cudaStream_t st, Grid ph, Grid pl, Grid ph2, Grid pl2, int n, int lo,
                        const double* mom, double S) {
  const long long P = ph.s + 2, tot = P * P * P;
  k_ball_ghosts<<<(int)((tot + 255) / 256), 256, 0, st>>>(ph, pl, ph2, pl2, n, lo, mom, S);
  note_launch();
}

// The same Dirichlet values into the ghost layer of an FP64 potential
// (PM_MIXED_FP64).
__global__ void __launch_bounds__(256) k_boundary64(GridD p, int n, int lo,
                                                    const double* __restrict__ mom, double S) {
  int i, j, k;
  if (!ghost_cell(blockIdx.x * (long long)blockDim.x + threadIdx.x, p.s, i, j, k)) return;
  p.base[(long long)i + (long long)j * p.sy + (long long)k * p.sz] =
      ghost_value(n, lo, i, j, k, mom, S);
}

void launch_boundary64(cudaStream_t st, GridD p, int n, int lo, const double* mom, double S) {
  long long tot = 6LL * (p.s + 2) * (p.s + 2);
  k_boundary64<<<(int)((tot + 255) / 256), 256, 0, st>>>(p, n, lo, mom, S);
  note_launch();
}

// ---------------------------------------------------------------------------
// Alternating-direction explicit half-substep (Sec. 2.3; Saul'yev form) of
// dPhi/dtau = D (lap Phi - f), lam = D dtau_sub:
//   Phi_c (1 + lam m_new) = Phi_c,old (1 - lam (6 - m_new)) + lam (sum_q Phi_q - fscale f)
// over a sweep of the cube in lexicographic order (upward or downward),
// Phi_q as it stands in memory (m_new of the six already swept).  The sweep
// runs as a wavefront: one launch per plane i + j + k = d, whose cells
// depend only on the planes before it; a cell's lower neighbours (upper when
// downward) lie on the plane before and its upper ones on the plane after,
// and across the periodic wrap the neighbour of a first cell lies on a later
// plane, that of a last cell on an earlier one -- exactly as in the
// sequential sweep, whose result this is.  FP64 arithmetic on the
// double-float potential; c_a[m] = 1 - lam (6 - m), c_b[m] = 1 / (1 + lam m).
// Open cubes: the ghost layer holds the Dirichlet values (read only).
// ---------------------------------------------------------------------------
struct AdeCoef {
  double a[7], b[7];
};

template <bool UP>
__device__ __forceinline__ void ade_cell(Grid ph, Grid pl, Grid fh, Grid fl, double fscale,
                                         double lam, const AdeCoef& cf, int periodic, int i,
                                         int j, int k) {
  const int s = ph.s;
  const int im = periodic ? (i == 0 ? s - 1 : i - 1) : i - 1;
  const int ip = periodic ? (i == s - 1 ? 0 : i + 1) : i + 1;
  const int jm = periodic ? (j == 0 ? s - 1 : j - 1) : j - 1;
  const int jp = periodic ? (j == s - 1 ? 0 : j + 1) : j + 1;
  const int km = periodic ? (k == 0 ? s - 1 : k - 1) : k - 1;
  const int kp = periodic ? (k == s - 1 ? 0 : k + 1) : k + 1;
  const int nb[6] = {gidx(ph, im, j, k), gidx(ph, ip, j, k), gidx(ph, i, jm, k),
                     gidx(ph, i, jp, k), gidx(ph, i, j, km), gidx(ph, i, j, kp)};
  int m_new = 3;
  if (periodic) {
    // swept before: upward the lower neighbour unless it wraps, and the upper
    // one when it wraps (mirror image downward)
    const int idx[3] = {i, j, k};
    m_new = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a)
      m_new += UP ? (idx[a] > 0) + (idx[a] == s - 1) : (idx[a] < s - 1) + (idx[a] == 0);
  }
  double sum = 0.0;
#pragma unroll
  for (int q = 0; q < 6; ++q) sum += (double)ph.base[nb[q]] + (double)pl.base[nb[q]];
  const int c = gidx(ph, i, j, k);
  const double old = (double)ph.base[c] + (double)pl.base[c];
  const int fc = gidx(fh, i, j, k);
  const double f = ((double)fh.base[fc] + (double)fl.base[fc]) * fscale;
  const double v = (cf.a[m_new] * old + lam * (sum - f)) * cf.b[m_new];
  const float h = (float)v;
  ph.base[c] = h;
  pl.base[c] = (float)(v - (double)h);
}

// The whole sweep in one cooperative launch: every thread takes its share of
// a plane's cells, then the grid waits (grid-wide barrier) before the next
// plane.  All blocks are resident (the launch is sized by the occupancy).
template <bool UP>
__global__ void __launch_bounds__(256) k_ade_sweep(Grid ph, Grid pl, Grid fh, Grid fl,
                                                   double fscale, double lam, AdeCoef cf,
                                                   int periodic) {
  cg::grid_group grid = cg::this_grid();
  const int s = ph.s, np = 3 * s - 2;
  const int stride = gridDim.x * blockDim.x;
  for (int q = 0; q < np; ++q) {
    const int d = UP ? q : np - 1 - q;
    // cells of the plane: j + k in [d - s + 1, d], i = d - j - k
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < s * s; t += stride) {
      const int j = t % s, k = t / s, i = d - j - k;
      if (i >= 0 && i < s) ade_cell<UP>(ph, pl, fh, fl, fscale, lam, cf, periodic, i, j, k);
    }
    grid.sync();
  }
}

cudaError_t launch_ade_sweep(cudaStream_t st, Grid ph, Grid pl, Grid fh, Grid fl,
                             double fscale, int periodic, double lam, bool upward) {
  AdeCoef cf;
  for (int m = 0; m <= 6; ++m) {
    cf.a[m] = 1.0 - lam * (6 - m);
    cf.b[m] = 1.0 / (1.0 + lam * m);
  }
  // resident blocks: queried once per direction
  static int per_sm[2] = {-1, -1};
  static int n_sm = 0;
  const int u = upward ? 1 : 0;
  if (per_sm[u] < 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm[u], upward ? (const void*)k_ade_sweep<true> : (const void*)k_ade_sweep<false>,
        256, 0);
    if (e != cudaSuccess) return e;
  }
  const int need = (ph.s * ph.s + 255) / 256;
  const int blocks = std::max(1, std::min(need, per_sm[u] * n_sm));
  void* args[] = {&ph, &pl, &fh, &fl, &fscale, &lam, &cf, &periodic};
  cudaError_t e = cudaLaunchCooperativeKernel(
      upward ? (const void*)k_ade_sweep<true> : (const void*)k_ade_sweep<false>,
      dim3((unsigned)blocks), dim3(256), args, 0, st);
  note_launch();
  return e;
}

// ---------------------------------------------------------------------------
// Batched forms.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) kb_deposit(const DepositDesc* d, const BTable* t) {
  int q;
  BI bi;
  if (!batch_map(d, t, (const int*)nullptr, q, bi)) return;
  const DepositDesc& e = d[q];
  d_drift_deposit<true>(bi, e.pos, e.mom, e.N, e.c0, e.n, e.lo, e.s, e.periodic, e.rho,
                        e.escaped);
}
__global__ void __launch_bounds__(256) kb_source(const SourceDesc* d, const BTable* t) {
  int q;
  BI bi;
  if (!batch_map(d, t, (const int*)nullptr, q, bi)) return;
  const SourceDesc& e = d[q];
  if (e.moments)
    d_source<true>(bi, e.rho, e.n, e.lo, e.s, e.fh, e.fl, e.invM, e.S, e.bgw, nullptr,
                   e.partial_f2,
                   (__int128*)e.partial_m, e.counter, e.out, e.bgm, e.invM_d, e.overflow);
  else
    d_source<false>(bi, e.rho, e.n, e.lo, e.s, e.fh, e.fl, e.invM, e.S, e.bgw, nullptr,
                    e.partial_f2, (__int128*)e.partial_m, e.counter, e.out, e.bgm, e.invM_d,
                    e.overflow);
}
__global__ void __launch_bounds__(256) kb_boundary(const BoundaryDesc* d, const BTable* t) {
  int q;
  BI bi;
  if (!batch_map(d, t, (const int*)nullptr, q, bi)) return;
  const BoundaryDesc& e = d[q];
  d_boundary(bi, e.ph, e.pl, e.n, e.lo, e.mom, e.S, e.want_lo, Grid{}, Grid{});
}

void launch_deposit_b(cudaStream_t st, int grid, const DepositDesc* d, const BTable* t) {
  if (grid <= 0) return;
  kb_deposit<<<grid, 256, 0, st>>>(d, t);
  note_launch();
}
void launch_source_b(cudaStream_t st, int grid, const SourceDesc* d, const BTable* t) {
  if (grid <= 0) return;
  kb_source<<<grid, dim3(32, 8), 0, st>>>(d, t);
  note_launch();
}
void launch_boundary_b(cudaStream_t st, int grid, const BoundaryDesc* d, const BTable* t) {
  if (grid <= 0) return;
  kb_boundary<<<grid, 256, 0, st>>>(d, t);
  note_launch();
}
int boundary_blocks(int s) { return (int)((6LL * (s + 2) * (s + 2) + 255) / 256); }
int deposit_blocks(long long N) {
  long long b = (N + 1023) / 1024 * 4;
  return (int)(b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b));
}

}  // namespace pm
