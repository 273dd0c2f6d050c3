// Geometric multigrid for the 7-point Poisson operator (Sec. 2.1, Eq. 3,
// cell units, h_l = 2^l on level l): red-black Gauss-Seidel smoothing,
// fused residual + 8-cell restriction, trilinear prolongation + correction,
// a single-CTA coarsest solve, and the double-float defect-correction loop
// (residual of the double-float potential; Phi += e).
#include "pm_kernels.cuh"

namespace pm {

// ---------------------------------------------------------------------------
// One colour of RB-GS: cells with (i+j+k) % 2 == color,
//   u = (sum_nb u - h^2 b) / 6.
// Thread layout: x over half a row (s even), y, z over rows.
// ---------------------------------------------------------------------------
// Open boundaries on coarse levels: the fine problem's error vanishes at the
// finest ghost-cell centre, half a fine cell outside the cube face.  On level
// l (spacing H = 2^l) the ghost centre lies H/2 outside the face, so a linear
// profile through that point gives ghost = -gam * (adjacent interior value)
// with gam = (H - 1) / (H + 1) (0 on the finest level, where the ghost layer
// holds the Dirichlet data itself).  Coarse ghosts are stored as zero and the
// -gam term is folded into the diagonal: 6 + gam * (number of ghost faces).
__device__ __forceinline__ float bnd_diag(int i, int j, int k, int s, float gam) {
  int nb = (i == 0) + (i == s - 1) + (j == 0) + (j == s - 1) + (k == 0) + (k == s - 1);
  return 6.0f + gam * (float)nb;
}

__global__ void __launch_bounds__(256) k_rbgs(Grid u, Grid b, float h2, int color,
                                              int periodic, float gam) {
  const int s = u.s;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  int k = blockIdx.z;
  if (t >= (s >> 1) || j >= s) return;
  int i = 2 * t + ((j + k + color) & 1);
  int c = gidx(u, i, j, k);
  int xm = wrap_m(i, s, periodic) - i, xp = wrap_p(i, s, periodic) - i;
  int ym = (wrap_m(j, s, periodic) - j) * u.sy, yp = (wrap_p(j, s, periodic) - j) * u.sy;
  int zm = (wrap_m(k, s, periodic) - k) * u.sz, zp = (wrap_p(k, s, periodic) - k) * u.sz;
  const float* p = u.base + c;
  float sum = (p[xm] + p[xp]) + (p[ym] + p[yp]) + (p[zm] + p[zp]);
  float bv = b.base[gidx(b, i, j, k)];
  if (periodic || gam == 0.0f)
    u.base[c] = (sum - h2 * bv) * (1.0f / 6.0f);
  else
    u.base[c] = (sum - h2 * bv) / bnd_diag(i, j, k, s, gam);
}

// ---------------------------------------------------------------------------
// Residual r = b - (sum_nb u - 6u)/h^2 on the 8 children of each coarse cell,
// averaged into the coarse right-hand side; the coarse unknown is zeroed.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_resid_restrict(Grid u, Grid b, float inv_h2,
                                                        Grid uc, Grid bc, int periodic,
                                                        float gam) {
  const int s = u.s;
  const int sc = uc.s;
  int I = blockIdx.x * blockDim.x + threadIdx.x;
  int J = blockIdx.y * blockDim.y + threadIdx.y;
  int K = blockIdx.z;
  if (I >= sc || J >= sc) return;
  float acc = 0.f;
#pragma unroll
  for (int dz = 0; dz < 2; ++dz)
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
      for (int dx = 0; dx < 2; ++dx) {
        int i = 2 * I + dx, j = 2 * J + dy, k = 2 * K + dz;
        int c = gidx(u, i, j, k);
        const float* p = u.base + c;
        int xm = wrap_m(i, s, periodic) - i, xp = wrap_p(i, s, periodic) - i;
        int ym = (wrap_m(j, s, periodic) - j) * u.sy, yp = (wrap_p(j, s, periodic) - j) * u.sy;
        int zm = (wrap_m(k, s, periodic) - k) * u.sz, zp = (wrap_p(k, s, periodic) - k) * u.sz;
        float diag = (periodic || gam == 0.0f) ? 6.0f : bnd_diag(i, j, k, s, gam);
        float lap = (p[xm] + p[xp]) + (p[ym] + p[yp]) + (p[zm] + p[zp]) - diag * p[0];
        acc += b.base[gidx(b, i, j, k)] - lap * inv_h2;
      }
  int cc = gidx(uc, I, J, K);
  bc.base[cc] = 0.125f * acc;
  uc.base[cc] = 0.0f;
}

// ---------------------------------------------------------------------------
// u += P uc: trilinear interpolation of the cell-centred coarse correction
// (weights 3/4 on the parent, 1/4 on the next coarse cell per axis).  Coarse
// ghosts are zero (open) or wrap (periodic).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_prolong(Grid uc, Grid u, int periodic,
                                                 float gam_c) {
  const int s = u.s;
  const int sc = uc.s;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  int k = blockIdx.z;
  if (i >= s || j >= s) return;
  int I = i >> 1, J = j >> 1, K = k >> 1;
  int I2 = (i & 1) ? I + 1 : I - 1;
  int J2 = (j & 1) ? J + 1 : J - 1;
  int K2 = (k & 1) ? K + 1 : K - 1;
  // open: a coarse ghost is -gam_c times the interior value beside it (per
  // axis), see bnd_diag
  float fx = 1.0f, fy = 1.0f, fz = 1.0f;
  if (periodic) {
    I2 = (I2 + sc) % sc;
    J2 = (J2 + sc) % sc;
    K2 = (K2 + sc) % sc;
  } else {
    if (I2 < 0 || I2 >= sc) { I2 = I; fx = -gam_c; }
    if (J2 < 0 || J2 >= sc) { J2 = J; fy = -gam_c; }
    if (K2 < 0 || K2 >= sc) { K2 = K; fz = -gam_c; }
  }
  const float* q = uc.base;
  float c000 = q[gidx(uc, I, J, K)], c100 = fx * q[gidx(uc, I2, J, K)];
  float c010 = fy * q[gidx(uc, I, J2, K)], c110 = fx * fy * q[gidx(uc, I2, J2, K)];
  float c001 = fz * q[gidx(uc, I, J, K2)], c101 = fx * fz * q[gidx(uc, I2, J, K2)];
  float c011 = fy * fz * q[gidx(uc, I, J2, K2)], c111 = fx * fy * fz * q[gidx(uc, I2, J2, K2)];
  float a0 = 0.75f * c000 + 0.25f * c100, a1 = 0.75f * c010 + 0.25f * c110;
  float a2 = 0.75f * c001 + 0.25f * c101, a3 = 0.75f * c011 + 0.25f * c111;
  float b0 = 0.75f * a0 + 0.25f * a1, b1 = 0.75f * a2 + 0.25f * a3;
  u.base[gidx(u, i, j, k)] += 0.75f * b0 + 0.25f * b1;
}

// ---------------------------------------------------------------------------
// Coarsest level (s <= 8): one CTA, RB-GS sweeps in shared memory.  Periodic:
// the right-hand side and the result are projected to zero mean.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(512) k_coarse(Grid u, Grid b, float h2, int periodic,
                                                int sweeps, float gam) {
  const int s = u.s;
  const int P = s + 2;
  __shared__ float su[10 * 10 * 10];
  __shared__ float sb[8 * 8 * 8];
  __shared__ float red[32];
  const int tid = threadIdx.x;
  const int ncell = s * s * s;
  for (int t = tid; t < P * P * P; t += blockDim.x) {
    int i = t % P - 1, j = (t / P) % P - 1, k = t / (P * P) - 1;
    su[t] = u.base[gidx(u, i, j, k)];
  }
  for (int t = tid; t < ncell; t += blockDim.x) {
    int i = t % s, j = (t / s) % s, k = t / (s * s);
    sb[t] = b.base[gidx(b, i, j, k)];
  }
  __syncthreads();
  if (periodic) {
    float v = 0.f;
    for (int t = tid; t < ncell; t += blockDim.x) v += sb[t];
    v = warp_sumf(v);
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    float mean = 0.f;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) mean += red[w];
    mean /= ncell;
    for (int t = tid; t < ncell; t += blockDim.x) sb[t] -= mean;
    __syncthreads();
  }
  // Odd sides (3): same-colour cells meet across the periodic wrap, so one
  // thread sweeps lexicographically to stay deterministic.
  const bool serial = (s & 1) != 0;
  for (int sw = 0; sw < sweeps; ++sw) {
    if (serial) {
      if (tid == 0) {
        for (int t = 0; t < ncell; ++t) {
          int i = t % s, j = (t / s) % s, k = t / (s * s);
          int im = periodic ? (i + s - 1) % s : i - 1, ip = periodic ? (i + 1) % s : i + 1;
          int jm = periodic ? (j + s - 1) % s : j - 1, jp = periodic ? (j + 1) % s : j + 1;
          int km = periodic ? (k + s - 1) % s : k - 1, kp = periodic ? (k + 1) % s : k + 1;
#define SU(a, b2, c2) su[((c2) + 1) * P * P + ((b2) + 1) * P + (a) + 1]
          float sum = SU(im, j, k) + SU(ip, j, k) + SU(i, jm, k) + SU(i, jp, k) +
                      SU(i, j, km) + SU(i, j, kp);
          SU(i, j, k) = (sum - h2 * sb[t]) / (periodic ? 6.0f : bnd_diag(i, j, k, s, gam));
#undef SU
        }
      }
      __syncthreads();
      continue;
    }
    for (int color = 0; color < 2; ++color) {
      for (int t = tid; t < ncell; t += blockDim.x) {
        int i = t % s, j = (t / s) % s, k = t / (s * s);
        if (((i + j + k) & 1) != color) continue;
        int im = periodic ? (i + s - 1) % s : i - 1, ip = periodic ? (i + 1) % s : i + 1;
        int jm = periodic ? (j + s - 1) % s : j - 1, jp = periodic ? (j + 1) % s : j + 1;
        int km = periodic ? (k + s - 1) % s : k - 1, kp = periodic ? (k + 1) % s : k + 1;
#define SU(a, b2, c2) su[((c2) + 1) * P * P + ((b2) + 1) * P + (a) + 1]
        float sum = SU(im, j, k) + SU(ip, j, k) + SU(i, jm, k) + SU(i, jp, k) +
                    SU(i, j, km) + SU(i, j, kp);
        SU(i, j, k) = (sum - h2 * sb[t]) / (periodic ? 6.0f : bnd_diag(i, j, k, s, gam));
#undef SU
      }
      __syncthreads();
    }
  }
  if (periodic) {
    float v = 0.f;
    for (int t = tid; t < ncell; t += blockDim.x) {
      int i = t % s, j = (t / s) % s, k = t / (s * s);
      v += su[(k + 1) * P * P + (j + 1) * P + i + 1];
    }
    v = warp_sumf(v);
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    float mean = 0.f;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) mean += red[w];
    mean /= ncell;
    for (int t = tid; t < ncell; t += blockDim.x) {
      int i = t % s, j = (t / s) % s, k = t / (s * s);
      su[(k + 1) * P * P + (j + 1) * P + i + 1] -= mean;
    }
    __syncthreads();
  }
  for (int t = tid; t < ncell; t += blockDim.x) {
    int i = t % s, j = (t / s) % s, k = t / (s * s);
    u.base[gidx(u, i, j, k)] = su[(k + 1) * P * P + (j + 1) * P + i + 1];
  }
}

static inline dim3 grid_half(int s) { return dim3((unsigned)((s / 2 + 31) / 32), (unsigned)((s + 7) / 8), (unsigned)s); }
static inline dim3 grid_full(int s) { return dim3((unsigned)((s + 31) / 32), (unsigned)((s + 7) / 8), (unsigned)s); }

void launch_rbgs(cudaStream_t st, Grid u, Grid b, float h2, int color, int periodic,
                 float gam) {
  k_rbgs<<<grid_half(u.s), dim3(32, 8), 0, st>>>(u, b, h2, color, periodic, gam);
  note_launch();
}
void launch_resid_restrict(cudaStream_t st, Grid u, Grid b, float inv_h2, Grid uc, Grid bc,
                           int periodic, float gam) {
  k_resid_restrict<<<grid_full(uc.s), dim3(32, 8), 0, st>>>(u, b, inv_h2, uc, bc, periodic,
                                                            gam);
  note_launch();
}
void launch_prolong(cudaStream_t st, Grid uc, Grid u, int periodic, float gam_c) {
  k_prolong<<<grid_full(u.s), dim3(32, 8), 0, st>>>(uc, u, periodic, gam_c);
  note_launch();
}
void launch_coarse(cudaStream_t st, Grid u, Grid b, float h2, int periodic, int sweeps,
                   float gam) {
  k_coarse<<<1, 512, 0, st>>>(u, b, h2, periodic, sweeps, gam);
  note_launch();
}

// ---------------------------------------------------------------------------
// Double-float defect: r = f - (sum_nb Phi - 6 Phi) with Phi = hi + lo and
// f = fh + fl.  The hi parts are summed by a TwoSum cascade, their rounding
// errors and the lo parts in a float compensation term (error ~ 2^-46 of
// the largest term).  Writes r (float) to the V-cycle right-hand side,
// zeroes the correction e, and reduces ||r||^2.  When phi is FP32 only
// (plain precision) the lo planes are all zero and the same kernel gives the
// residual of the FP32 potential.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_defect(Grid ph, Grid pl, Grid fh, Grid fl, Grid rb,
                                                Grid e, int periodic, int write_r,
                                                double* __restrict__ partial,
                                                unsigned int* counter, double* __restrict__ out) {
  const int s = ph.s;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  float r2 = 0.f;
  for (int k = blockIdx.z; k < s && i < s && j < s; k += gridDim.z) {
    int c = gidx(ph, i, j, k);
    int xm = wrap_m(i, s, periodic) - i, xp = wrap_p(i, s, periodic) - i;
    int ym = (wrap_m(j, s, periodic) - j) * ph.sy, yp = (wrap_p(j, s, periodic) - j) * ph.sy;
    int zm = (wrap_m(k, s, periodic) - k) * ph.sz, zp = (wrap_p(k, s, periodic) - k) * ph.sz;
    const float* h = ph.base + c;
    const float* l = pl.base + c;
    int fc = gidx(fh, i, j, k);
    // r = f - sum_nb + 6 phi
    float sacc = fh.base[fc];
    float comp = fl.base[fc];
    df t;
    t = two_sum(sacc, -h[xm]); sacc = t.hi; comp += t.lo;
    t = two_sum(sacc, -h[xp]); sacc = t.hi; comp += t.lo;
    t = two_sum(sacc, -h[ym]); sacc = t.hi; comp += t.lo;
    t = two_sum(sacc, -h[yp]); sacc = t.hi; comp += t.lo;
    t = two_sum(sacc, -h[zm]); sacc = t.hi; comp += t.lo;
    t = two_sum(sacc, -h[zp]); sacc = t.hi; comp += t.lo;
    df p6 = two_prod(6.0f, h[0]);
    t = two_sum(sacc, p6.hi); sacc = t.hi; comp += t.lo + p6.lo;
    comp -= (l[xm] + l[xp]) + (l[ym] + l[yp]) + (l[zm] + l[zp]);
    comp += 6.0f * l[0];
    float r = sacc + comp;
    if (write_r) {
      int rc = gidx(rb, i, j, k);
      rb.base[rc] = r;
      e.base[gidx(e, i, j, k)] = 0.0f;
    }
    r2 = __fmaf_rn(r, r, r2);
  }
  __shared__ double sm[32];
  double v = warp_sum((double)r2);
  int lane = (threadIdx.y * blockDim.x + threadIdx.x) & 31;
  int warp = (threadIdx.y * blockDim.x + threadIdx.x) >> 5;
  if (lane == 0) sm[warp] = v;
  __syncthreads();
  unsigned nblk = gridDim.x * gridDim.y * gridDim.z;
  unsigned bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
  __shared__ bool last;
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    double tb = 0.0;
    int nw = (blockDim.x * blockDim.y) >> 5;
    for (int w = 0; w < nw; ++w) tb += sm[w];
    partial[bid] = tb;
    __threadfence();
    unsigned tk = atomicAdd(counter, 1u);
    last = (tk == nblk - 1);
  }
  __syncthreads();
  if (!last) return;
  int tid = threadIdx.y * blockDim.x + threadIdx.x;
  int nth = blockDim.x * blockDim.y;
  double acc = 0.0;
  for (unsigned q = tid; q < nblk; q += nth) acc += __ldcg(partial + q);
  acc = warp_sum(acc);
  __syncthreads();
  if (lane == 0) sm[warp] = acc;
  __syncthreads();
  if (tid == 0) {
    double tt = 0.0;
    for (int w = 0; w < nth / 32; ++w) tt += sm[w];
    *out = tt;
    *counter = 0u;
  }
}

static inline dim3 grid_defect(int s) {
  return dim3((unsigned)((s + 31) / 32), (unsigned)((s + 7) / 8), (unsigned)(s < 16 ? s : 16));
}
int defect_blocks(int s) {
  dim3 g = grid_defect(s);
  return (int)(g.x * g.y * g.z);
}

void launch_defect(cudaStream_t st, Grid ph, Grid pl, Grid fh, Grid fl, Grid rb, Grid e,
                   int periodic, bool write_r, double* partial, unsigned int* counter,
                   double* out) {
  k_defect<<<grid_defect(ph.s), dim3(32, 8), 0, st>>>(ph, pl, fh, fl, rb, e, periodic,
                                                    write_r ? 1 : 0, partial, counter, out);
  note_launch();
}

// Phi (hi, lo) += e.
__global__ void __launch_bounds__(256) k_correct(Grid ph, Grid pl, Grid e) {
  const int s = ph.s;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  int k = blockIdx.z;
  if (i >= s || j >= s) return;
  int c = gidx(ph, i, j, k);
  df v = df_add(df{ph.base[c], pl.base[c]}, df{e.base[gidx(e, i, j, k)], 0.0f});
  ph.base[c] = v.hi;
  pl.base[c] = v.lo;
}

void launch_correct(cudaStream_t st, Grid ph, Grid pl, Grid e) {
  k_correct<<<grid_full(ph.s), dim3(32, 8), 0, st>>>(ph, pl, e);
  note_launch();
}

// Fill the interior (and optionally the ghost layer) of a grid with v.
__global__ void k_fill(Grid g, float v, int with_ghost) {
  int gs = g.s + (with_ghost ? 2 : 0);
  int off = with_ghost ? -1 : 0;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  int k = blockIdx.z;
  if (i >= gs || j >= gs) return;
  g.base[gidx(g, i + off, j + off, k + off)] = v;
}

void launch_fill(cudaStream_t st, Grid g, float v, bool with_ghost) {
  int gs = g.s + (with_ghost ? 2 : 0);
  k_fill<<<grid_full(gs), dim3(32, 8), 0, st>>>(g, v, with_ghost ? 1 : 0);
  note_launch();
}

// Potential output of pm_potential: phi32 = hi, phi64 = hi + lo (optional),
// periodic results shifted by -mean (mean given as hi+lo sums).
__global__ void k_phi_out(Grid ph, Grid pl, float* out32, double* out64, double shift) {
  const int s = ph.s;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  int k = blockIdx.z;
  if (i >= s || j >= s) return;
  int c = gidx(ph, i, j, k);
  double v = (double)ph.base[c] + (double)pl.base[c] - shift;
  long long o = ((long long)k * s + j) * s + i;
  out32[o] = (float)v;
  if (out64) out64[o] = v;
}

void launch_phi_out(cudaStream_t st, Grid ph, Grid pl, float* out32, double* out64,
                    double shift) {
  k_phi_out<<<grid_full(ph.s), dim3(32, 8), 0, st>>>(ph, pl, out32, out64, shift);
  note_launch();
}

// Sum of hi + lo over the interior (for the periodic zero-mean gauge); FP64
// per thread, not on the step's hot path.
__global__ void k_sum_phi(Grid ph, Grid pl, double* __restrict__ partial,
                          unsigned int* counter, double* __restrict__ out) {
  const int s = ph.s;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  double v = 0.0;
  for (int k = blockIdx.z; k < s && i < s && j < s; k += gridDim.z) {
    int c = gidx(ph, i, j, k);
    v += (double)ph.base[c] + (double)pl.base[c];
  }
  __shared__ double sm[32];
  int tid = threadIdx.y * blockDim.x + threadIdx.x;
  v = warp_sum(v);
  if ((tid & 31) == 0) sm[tid >> 5] = v;
  __syncthreads();
  unsigned nblk = gridDim.x * gridDim.y * gridDim.z;
  unsigned bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
  __shared__ bool last;
  if (tid == 0) {
    double tb = 0.0;
    for (int w = 0; w < (int)(blockDim.x * blockDim.y) / 32; ++w) tb += sm[w];
    partial[bid] = tb;
    __threadfence();
    last = (atomicAdd(counter, 1u) == nblk - 1);
  }
  __syncthreads();
  if (!last || tid != 0) return;
  double tt = 0.0;
  for (unsigned q = 0; q < nblk; ++q) tt += __ldcg(partial + q);
  *out = tt;
  *counter = 0u;
}

void launch_sum_phi(cudaStream_t st, Grid ph, Grid pl, double* partial, unsigned int* counter,
                    double* out) {
  k_sum_phi<<<grid_defect(ph.s), dim3(32, 8), 0, st>>>(ph, pl, partial, counter, out);
  note_launch();
}

}  // namespace pm
