// FP64 everywhere (precision PM_FP64_PLAIN): the Poisson solve of Eq. 3
// with the potential, the source and every multigrid level in double, the
// same V(2,2) cycle as the FP32 path (red-black SOR, 8-cell
// average restriction of the residual, trilinear prolongation, the
// coarse-level open-boundary factor folded into the diagonal) and a one-CTA
// bottom.  It exists to measure what FP64 costs on this GPU against the
// double-float defect correction; results are converted from and to the
// double-float pair the rest of the step uses.
#include "pm_kernels.cuh"

namespace pm {

namespace {
__device__ __forceinline__ long long gidxd(const GridD& g, int i, int j, int k) {
  return (long long)i + (long long)j * g.sy + (long long)k * g.sz;
}
__device__ __forceinline__ double diag64(int i, int j, int k, int s, int periodic, double gam) {
  if (periodic) return 6.0;
  const int nb = (i == 0) + (i == s - 1) + (j == 0) + (j == s - 1) + (k == 0) + (k == s - 1);
  return 6.0 + gam * (double)nb;
}
__device__ __forceinline__ int wm(int i, int s, int periodic) {
  return (i == 0 && periodic) ? s - 1 : i - 1;
}
__device__ __forceinline__ int wp(int i, int s, int periodic) {
  return (i == s - 1 && periodic) ? 0 : i + 1;
}
// sum of the six neighbours of (i, j, k)
__device__ __forceinline__ double nbsum64(const GridD& u, int i, int j, int k, int periodic) {
  const int s = u.s;
  const double* p = u.base;
  return p[gidxd(u, wm(i, s, periodic), j, k)] + p[gidxd(u, wp(i, s, periodic), j, k)] +
         p[gidxd(u, i, wm(j, s, periodic), k)] + p[gidxd(u, i, wp(j, s, periodic), k)] +
         p[gidxd(u, i, j, wm(k, s, periodic))] + p[gidxd(u, i, j, wp(k, s, periodic))];
}
}  // namespace

// one colour of red-black SOR, u = u + omega ((sum_nb u - h^2 b) / diag - u),
// cells (i+j+k) % 2 == color, omega = MG_OMEGA as in the FP32 forms
__global__ void __launch_bounds__(256) k64_rbgs(GridD u, GridD b, double h2, int color,
                                                int periodic, double gam) {
  const int s = u.s;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y, k = blockIdx.z;
  if (j >= s) return;
  const int i = 2 * t + ((j + k + color) & 1);
  if (i >= s) return;
  const double gs = (nbsum64(u, i, j, k, periodic) - h2 * b.base[gidxd(b, i, j, k)]) /
                    diag64(i, j, k, s, periodic, gam);
  double* c = u.base + gidxd(u, i, j, k);
  *c = *c + (double)MG_OMEGA * (gs - *c);
}

// coarse b = average over the 8 children of r = b - (sum_nb u - diag u) / h^2;
// the coarse iterate is zeroed
__global__ void __launch_bounds__(256) k64_resid_restrict(GridD u, GridD b, double inv_h2,
                                                          GridD uc, GridD bc, int periodic,
                                                          double gam) {
  const int s = u.s, sc = uc.s;
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y, K = blockIdx.z;
  if (I >= sc || J >= sc) return;
  double acc = 0.0;
  for (int dz = 0; dz < 2; ++dz)
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) {
        const int i = 2 * I + dx, j = 2 * J + dy, k = 2 * K + dz;
        const double uc0 = u.base[gidxd(u, i, j, k)];
        const double lap = nbsum64(u, i, j, k, periodic) - diag64(i, j, k, s, periodic, gam) * uc0;
        acc += b.base[gidxd(b, i, j, k)] - lap * inv_h2;
      }
  const long long c = gidxd(uc, I, J, K);
  bc.base[c] = 0.125 * acc;
  uc.base[c] = 0.0;
}

// u += P uc: weights 3/4 on the parent and 1/4 on the next coarse cell per
// axis; an open coarse ghost is -gam_c times the interior value beside it
__global__ void __launch_bounds__(256) k64_prolong(GridD uc, GridD u, int periodic,
                                                   double gam_c) {
  const int s = u.s, sc = uc.s;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y, k = blockIdx.z;
  if (i >= s || j >= s) return;
  const int I = i >> 1, J = j >> 1, K = k >> 1;
  int I2 = (i & 1) ? I + 1 : I - 1, J2 = (j & 1) ? J + 1 : J - 1, K2 = (k & 1) ? K + 1 : K - 1;
  double fx = 1.0, fy = 1.0, fz = 1.0;
  if (periodic) {
    I2 = I2 < 0 ? sc - 1 : (I2 >= sc ? 0 : I2);
    J2 = J2 < 0 ? sc - 1 : (J2 >= sc ? 0 : J2);
    K2 = K2 < 0 ? sc - 1 : (K2 >= sc ? 0 : K2);
  } else {
    if (I2 < 0 || I2 >= sc) { I2 = I; fx = -gam_c; }
    if (J2 < 0 || J2 >= sc) { J2 = J; fy = -gam_c; }
    if (K2 < 0 || K2 >= sc) { K2 = K; fz = -gam_c; }
  }
  const double* q = uc.base;
  auto l34 = [](double a, double b2) { return 0.75 * a + 0.25 * b2; };
  const double a0 = l34(q[gidxd(uc, I, J, K)], fx * q[gidxd(uc, I2, J, K)]);
  const double a1 = l34(fy * q[gidxd(uc, I, J2, K)], fx * fy * q[gidxd(uc, I2, J2, K)]);
  const double a2 = l34(fz * q[gidxd(uc, I, J, K2)], fx * fz * q[gidxd(uc, I2, J, K2)]);
  const double a3 = l34(fy * fz * q[gidxd(uc, I, J2, K2)], fx * fy * fz * q[gidxd(uc, I2, J2, K2)]);
  u.base[gidxd(u, i, j, k)] += l34(l34(a0, a1), l34(a2, a3));
}

// the coarsest level in one CTA: `sweeps` red-black sweeps (lexicographic in
// one thread on an odd periodic side, where red-black does not close over
// the wrap); the iterate starts at the zero the restriction left
__global__ void __launch_bounds__(256) k64_bottom(GridD u, GridD b, double h2, int periodic,
                                                  double gam, int sweeps) {
  const int s = u.s, n3 = s * s * s;
  auto upd = [&](int i, int j, int k) {
    u.base[gidxd(u, i, j, k)] =
        (nbsum64(u, i, j, k, periodic) - h2 * b.base[gidxd(b, i, j, k)]) /
        diag64(i, j, k, s, periodic, gam);
  };
  if (periodic && (s & 1)) {
    if (threadIdx.x == 0)
      for (int sw = 0; sw < sweeps; ++sw)
        for (int k = 0; k < s; ++k)
          for (int j = 0; j < s; ++j)
            for (int i = 0; i < s; ++i) upd(i, j, k);
    return;
  }
  for (int sw = 0; sw < sweeps; ++sw)
    for (int color = 0; color < 2; ++color) {
      for (int c = threadIdx.x; c < n3; c += blockDim.x) {
        const int i = c % s, j = (c / s) % s, k = c / (s * s);
        if (((i + j + k) & 1) == color) upd(i, j, k);
      }
      __syncthreads();
    }
}

// ||f - (sum_nb Phi - 6 Phi)||^2 over the interior (level 0: the ghost layer
// holds the Dirichlet data, or the grid wraps); block sums in partial[], the
// last block adds them in block order into *out and clears the counter
__global__ void __launch_bounds__(256) k64_defect(GridD p, GridD f, int periodic,
                                                  double* __restrict__ partial,
                                                  unsigned int* counter, double* __restrict__ out) {
  const int s = p.s;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int chunk = (s + gridDim.z - 1) / gridDim.z;
  const int k0 = blockIdx.z * chunk, k1 = min(s, k0 + chunk);
  double r2 = 0.0;
  if (i < s && j < s)
    for (int k = k0; k < k1; ++k) {
      const double r = f.base[gidxd(f, i, j, k)] -
                       (nbsum64(p, i, j, k, periodic) - 6.0 * p.base[gidxd(p, i, j, k)]);
      r2 += r * r;
    }
  __shared__ double sm[8];
  __shared__ bool last;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const double w = warp_sum(r2);
  if (lane == 0) sm[warp] = w;
  __syncthreads();
  const unsigned nblk = gridDim.x * gridDim.y * gridDim.z;
  const unsigned bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
  if (tid == 0) {
    double t = 0.0;
    for (int q = 0; q < 8; ++q) t += sm[q];
    partial[bid] = t;
    __threadfence();
    last = atomicAdd(counter, 1u) == nblk - 1;
  }
  __syncthreads();
  if (!last) return;
  double acc = 0.0;
  for (unsigned q = tid; q < nblk; q += 256) acc += __ldcg(partial + q);
  acc = warp_sum(acc);
  __syncthreads();
  if (lane == 0) sm[warp] = acc;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int q = 0; q < 8; ++q) t += sm[q];
    *out = t;
    *counter = 0u;
  }
}

// out = hi + lo in double over the interior, or also the ghost layer
__global__ void __launch_bounds__(256) k64_from_pair(Grid hi, Grid lo, GridD out, int ghost) {
  const int g = ghost ? 1 : 0, m = hi.s + 2 * g;
  const int a = blockIdx.x * blockDim.x + threadIdx.x, c = blockIdx.y * blockDim.y + threadIdx.y;
  if (a >= m || c >= m) return;
  const int i = a - g, j = c - g, k = (int)blockIdx.z - g;
  const int q = gidx(hi, i, j, k);
  out.base[gidxd(out, i, j, k)] = (double)hi.base[q] + (double)lo.base[gidx(lo, i, j, k)];
}

// hi = fl(v), lo = fl(v - hi) over the interior, or also the ghost layer
__global__ void __launch_bounds__(256) k64_to_pair(GridD in, Grid hi, Grid lo, int ghost) {
  const int g = ghost ? 1 : 0, m = in.s + 2 * g;
  const int a = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y * blockDim.y + threadIdx.y;
  if (a >= m || b >= m) return;
  const int i = a - g, j = b - g, k = (int)blockIdx.z - g;
  const double v = in.base[gidxd(in, i, j, k)];
  const float h = (float)v;
  hi.base[gidx(hi, i, j, k)] = h;
  lo.base[gidx(lo, i, j, k)] = (float)(v - (double)h);
}

// ---------------------------------------------------------------------------
// Mixed precision with an FP64 outer loop (PM_MIXED_FP64): the potential
// stays in FP64 for the whole run; each V-cycle (FP32) solves A e = r for
// the residual r of the FP64 defect below, and the correction is added to
// the FP64 potential.
// ---------------------------------------------------------------------------

// Phi += e over the interior (e: the FP32 correction of the last V-cycle)
__global__ void __launch_bounds__(256) k64_correct(GridD p, Grid e) {
  pdl_wait();
  pdl_release();
  const int s = p.s;
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= s || j >= s) return;
  p.base[gidxd(p, i, j, k)] += (double)e.base[gidx(e, i, j, k)];
}

// r = f - (sum_nb Phi - 6 Phi) in FP64 at every interior cell (ghost layer:
// Dirichlet data, or the grid wraps), stored rounded to FP32 in rb (the
// V-cycle's right-hand side).  ||r||^2 of the stored values: per thread in
// FP32 over its run of planes, then in FP64; the last block adds the block
// sums in block order into *out.  Each thread walks a run of planes and
// rolls its column's z neighbours through registers.
__global__ void __launch_bounds__(256) k64m_defect(GridD p, GridD f, Grid rb, int periodic,
                                                   double* __restrict__ partial,
                                                   unsigned int* counter,
                                                   double* __restrict__ out) {
  pdl_wait();
  pdl_release();
  const int s = p.s;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int chunk = (s + gridDim.z - 1) / gridDim.z;
  const int k0 = blockIdx.z * chunk, k1 = min(s, k0 + chunk);
  float r2 = 0.0f;
  if (i < s && j < s && k0 < k1) {
    const double* P = p.base;
    const long long dxm = wm(i, s, periodic) - i, dxp = wp(i, s, periodic) - i;
    const long long dym = (long long)(wm(j, s, periodic) - j) * p.sy;
    const long long dyp = (long long)(wp(j, s, periodic) - j) * p.sy;
    double zm = P[gidxd(p, i, j, wm(k0, s, periodic))];
    double zc = P[gidxd(p, i, j, k0)];
    // the z+ neighbour is loaded one plane ahead of its use
    double zp = P[gidxd(p, i, j, wp(k0, s, periodic))];
    for (int k = k0; k < k1; ++k) {
      const long long c = gidxd(p, i, j, k);
      double zn = 0.0;
      if (k + 1 < k1) zn = P[gidxd(p, i, j, wp(k + 1, s, periodic))];  // plane k + 2 <= k1 <= s
      const double nb = ((P[c + dxm] + P[c + dxp]) + (P[c + dym] + P[c + dyp])) + (zm + zp);
      const double r = fma(6.0, zc, f.base[gidxd(f, i, j, k)]) - nb;
      const float r32 = (float)r;
      rb.base[gidx(rb, i, j, k)] = r32;
      r2 = fmaf(r32, r32, r2);
      zm = zc;
      zc = zp;
      zp = zn;
    }
  }
  __shared__ double sm[8];
  __shared__ bool last;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const double w = warp_sum((double)r2);
  if (lane == 0) sm[warp] = w;
  __syncthreads();
  const unsigned nblk = gridDim.x * gridDim.y * gridDim.z;
  const unsigned bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
  if (tid == 0) {
    double t = 0.0;
    for (int q = 0; q < 8; ++q) t += sm[q];
    partial[bid] = t;
    __threadfence();
    last = atomicAdd(counter, 1u) == nblk - 1;
  }
  __syncthreads();
  if (!last) return;
  double acc = 0.0;
  for (unsigned q = tid; q < nblk; q += 256) acc += __ldcg(partial + q);
  acc = warp_sum(acc);
  __syncthreads();
  if (lane == 0) sm[warp] = acc;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int q = 0; q < 8; ++q) t += sm[q];
    *out = t;
    *counter = 0u;
  }
}

// warm start extrapolated in time, Phi <- Phi + w (Phi - Phi_prev),
// Phi_prev <- old Phi (interior; the ghost layer keeps its boundary values)
__global__ void __launch_bounds__(256) k64_predict(GridD p, GridD q, double w) {
  pdl_wait();
  pdl_release();
  const int s = p.s;
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= s || j >= s) return;
  const long long c = gidxd(p, i, j, k);
  const double cur = p.base[c], prev = q.base[c];
  q.base[c] = cur;
  p.base[c] = cur + (cur - prev) * w;
}

// the interior set to v
__global__ void __launch_bounds__(256) k64_fill(GridD p, double v) {
  const int s = p.s;
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= s || j >= s) return;
  p.base[gidxd(p, i, j, blockIdx.z)] = v;
}

// G(c) = (gx, gy, gz, 0): centred differences of the FP64 potential at every
// cell of the active cube, rounded to FP32 (the gather's gradient field),
// in the full (n+2)^3 layout
__global__ void __launch_bounds__(256) k64_grad(const double* __restrict__ ph, int n, int lo,
                                                int s, int periodic, float4* __restrict__ G) {
  pdl_wait();
  pdl_release();
  const int P = n + 2;
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= s || j >= s) return;
  const int X = lo + i, Y = lo + j, Z = lo + k;
  auto w = [&](int a) { return periodic ? (a < 0 ? a + n : (a >= n ? a - n : a)) : a; };
  auto at = [&](int x, int y, int z) {
    return __ldg(ph + ((long long)(z + 1) * P + (y + 1)) * P + (x + 1));
  };
  const long long c = ((long long)(Z + 1) * P + (Y + 1)) * P + (X + 1);
  G[c] = make_float4((float)(at(w(X + 1), Y, Z) - at(w(X - 1), Y, Z)),
                     (float)(at(X, w(Y + 1), Z) - at(X, w(Y - 1), Z)),
                     (float)(at(X, Y, w(Z + 1)) - at(X, Y, w(Z - 1))), 0.0f);
}

namespace {
dim3 g64_full(int s) { return dim3((unsigned)((s + 31) / 32), (unsigned)((s + 7) / 8), (unsigned)s); }
}  // namespace

void launch64_rbgs(cudaStream_t st, GridD u, GridD b, double h2, int color, int periodic,
                   double gam) {
  const int half = (u.s + 1) / 2;
  k64_rbgs<<<dim3((unsigned)((half + 31) / 32), (unsigned)((u.s + 7) / 8), (unsigned)u.s),
             dim3(32, 8), 0, st>>>(u, b, h2, color, periodic, gam);
  note_launch();
}
void launch64_resid_restrict(cudaStream_t st, GridD u, GridD b, double inv_h2, GridD uc,
                             GridD bc, int periodic, double gam) {
  k64_resid_restrict<<<g64_full(uc.s), dim3(32, 8), 0, st>>>(u, b, inv_h2, uc, bc, periodic, gam);
  note_launch();
}
void launch64_prolong(cudaStream_t st, GridD uc, GridD u, int periodic, double gam_c) {
  k64_prolong<<<g64_full(u.s), dim3(32, 8), 0, st>>>(uc, u, periodic, gam_c);
  note_launch();
}
void launch64_bottom(cudaStream_t st, GridD u, GridD b, double h2, int periodic, double gam,
                     int sweeps) {
  k64_bottom<<<1, 256, 0, st>>>(u, b, h2, periodic, gam, sweeps);
  note_launch();
}
int defect64_blocks(int s) {
  return ((s + 31) / 32) * ((s + 7) / 8) * (s < 16 ? s : 16);
}
void launch64_defect(cudaStream_t st, GridD p, GridD f, int periodic, double* partial,
                     unsigned int* counter, double* out) {
  const int s = p.s;
  k64_defect<<<dim3((unsigned)((s + 31) / 32), (unsigned)((s + 7) / 8), (unsigned)(s < 16 ? s : 16)),
               dim3(32, 8), 0, st>>>(p, f, periodic, partial, counter, out);
  note_launch();
}
void launch64_from_pair(cudaStream_t st, Grid hi, Grid lo, GridD out, bool ghost) {
  const int m = hi.s + (ghost ? 2 : 0);
  k64_from_pair<<<g64_full(m), dim3(32, 8), 0, st>>>(hi, lo, out, ghost ? 1 : 0);
  note_launch();
}
void launch64_to_pair(cudaStream_t st, GridD in, Grid hi, Grid lo, bool ghost) {
  const int m = in.s + (ghost ? 2 : 0);
  k64_to_pair<<<g64_full(m), dim3(32, 8), 0, st>>>(in, hi, lo, ghost ? 1 : 0);
  note_launch();
}
void launch64_correct(cudaStream_t st, GridD p, Grid e) {
  launch_pdl(k64_correct, g64_full(p.s), dim3(32, 8), 0, st, p, e);
  note_launch();
}
void launch64m_defect(cudaStream_t st, GridD p, GridD f, Grid rb, int periodic, double* partial,
                      unsigned int* counter, double* out) {
  const int s = p.s;
  launch_pdl(k64m_defect, dim3((unsigned)((s + 31) / 32), (unsigned)((s + 7) / 8),
                               (unsigned)(s < 16 ? s : 16)),
             dim3(32, 8), 0, st, p, f, rb, periodic, partial, counter, out);
  note_launch();
}
void launch64_predict(cudaStream_t st, GridD p, GridD q, double w) {
  launch_pdl(k64_predict, g64_full(p.s), dim3(32, 8), 0, st, p, q, w);
  note_launch();
}
void launch64_fill(cudaStream_t st, GridD p, double v) {
  k64_fill<<<g64_full(p.s), dim3(32, 8), 0, st>>>(p, v);
  note_launch();
}
void launch64_grad(cudaStream_t st, const double* ph, int n, int lo, int s, int periodic,
                   float4* G) {
  launch_pdl(k64_grad, g64_full(s), dim3(32, 8), 0, st, ph, n, lo, s, periodic, G);
  note_launch();
}

}  // namespace pm
