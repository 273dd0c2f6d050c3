// Geometric multigrid for the 7-point Poisson operator (Sec. 2.1, Eq. 3,
// cell units, h_l = 2^l on level l): red-black SOR smoothing,
// fused residual + 8-cell restriction, trilinear prolongation + correction,
// a single-CTA coarsest solve, and the double-float defect-correction loop
// (residual of the double-float potential; Phi += e).
#include <cstdlib>

#include "cmg_dev.cuh"
#include "cmg_fast.cuh"
#include "mg_arith.cuh"
#include "pm_kernels.cuh"

namespace pm {

// ---------------------------------------------------------------------------
// One colour of red-black SOR: cells with (i+j+k) % 2 == color,
//   u = u + MG_OMEGA ((sum_nb u - h^2 b) / 6 - u).
// Thread layout: x over half a row (s even), y, z over rows.
// ---------------------------------------------------------------------------
// zero_start 1 (the first red sweep): the iterate is known to be zero, so
// the red cells take MG_OMEGA (-h^2 b)/diag without reading u; 2 (the black
// sweep after it): the black cells' own values are known to be zero (it
// reads only red neighbours), so u needs no clearing before a V-cycle.
// MASK: the ball solve's masked grids (compiled out of the unmasked form)
template <bool MASK>
__device__ __forceinline__ void d_rbgs(const BI& bi, Grid u, Grid b, float h2, int color,
                                              int periodic, float gam, int zero_start,
                                              float d0){
  // each thread updates the two cells of its colour at i0 and i0 + 2
  // (independent loads in flight, the shared x-neighbour loaded once)
  const int s = u.s;
  int t = bi.x * blockDim.x + threadIdx.x;
  int j = bi.y * blockDim.y + threadIdx.y;
  int k = bi.z;
  const int half = s >> 1;
  if (2 * t >= half || j >= s) return;
  const int i0 = 4 * t + ((j + k + color) & 1);
  const bool two = 2 * t + 1 < half;
  // the ball solve updates only the cells of its mask
  const bool in0 = !MASK || g_in(u, i0, j, k), in1 = two && (!MASK || g_in(u, i0 + 2, j, k));
  if (MASK && !in0 && !in1) return;
  const int ym = (wrap_m(j, s, periodic) - j) * u.sy, yp = (wrap_p(j, s, periodic) - j) * u.sy;
  const int zm = (wrap_m(k, s, periodic) - k) * u.sz, zp = (wrap_p(k, s, periodic) - k) * u.sz;
  // masked coarse levels of the ball solve: their own diagonal
  const bool ballc = MASK && ball_coarse(u);
  const bool simple = mg_simple(periodic, gam, d0) && !ballc;
  const int c0 = gidx(u, i0, j, k);
  const int bc0 = gidx(b, i0, j, k);
  float* p0 = u.base + c0;
  const float* bb = b.base + bc0;
  float b0v = bb[0], b1v = two ? bb[2] : 0.0f;
  float s0 = 0.0f, s1 = 0.0f;
  float o0 = 0.0f, o1 = 0.0f;  // the cells' old values (zero unless zero_start == 0)
  if (zero_start == 0) {
    o0 = p0[0];
    if (two) o1 = p0[2];
  }
  if (zero_start != 1) {  // (1: the neighbours are zero too)
    const int xm = wrap_m(i0, s, periodic) - i0;
    const int xp = wrap_p(i0, s, periodic) - i0;  // 1 unless i0 = s - 1 (then no i0 + 2)
    float xmid = p0[xp];  // right neighbour of i0, left of i0 + 2
    s0 = nb6(p0[xm], xmid, p0[ym], p0[yp], p0[zm], p0[zp]);
    if (two) {
      const int i1 = i0 + 2;
      const int xp1 = wrap_p(i1, s, periodic) - i1;
      float* p1 = p0 + 2;
      s1 = nb6(xmid, p1[xp1], p1[ym], p1[yp], p1[zm], p1[zp]);
    }
  }
  auto dg = [&](int i) {
    return simple ? 6.0f : (ballc ? ball_diag(u, i, j, k) : mg_diag(i, j, k, s, periodic, gam, d0));
  };
  if (in0) p0[0] = sor_value(o0, gs_value(s0, b0v, h2, simple, dg(i0)));
  if (in1) p0[2] = sor_value(o1, gs_value(s1, b1v, h2, simple, dg(i0 + 2)));
}

template <bool MASK>
__global__ void __launch_bounds__(256) k_rbgs(Grid u, Grid b, float h2, int color,
                                              int periodic, float gam, int zero_start, float d0) {
  pdl_wait();
  pdl_release();
  d_rbgs<MASK>(bi_native(), u, b, h2, color, periodic, gam, zero_start, d0);
}

// ---------------------------------------------------------------------------
// Residual r = b - (sum_nb u - 6u)/h^2 on the 8 children of each coarse cell,
// averaged into the coarse right-hand side; the coarse unknown is zeroed.
// ---------------------------------------------------------------------------
template <bool MASK>
__device__ __forceinline__ void d_resid_restrict(const BI& bi, Grid u, Grid b, float inv_h2,
                                                        Grid uc, Grid bc, int periodic,
                                                        float gam, float d0){
  const int s = u.s;
  const int sc = uc.s;
  int I = bi.x * blockDim.x + threadIdx.x;
  int J = bi.y * blockDim.y + threadIdx.y;
  int K = bi.z;
  if (I >= sc || J >= sc) return;
  // fine coordinates 2c-1 .. 2c+2 along each axis (wrapped, or the ghost
  // layer), as offsets
  const int i0 = 2 * I, j0 = 2 * J, k0 = 2 * K;
  const int xo[4] = {wrap_m(i0, s, periodic), i0, i0 + 1, wrap_p(i0 + 1, s, periodic)};
  const int yo[4] = {wrap_m(j0, s, periodic) * u.sy, j0 * u.sy, (j0 + 1) * u.sy,
                     wrap_p(j0 + 1, s, periodic) * u.sy};
  const int zo[4] = {wrap_m(k0, s, periodic) * u.sz, k0 * u.sz, (k0 + 1) * u.sz,
                     wrap_p(k0 + 1, s, periodic) * u.sz};
  const float* p = u.base;
  // the 8 children and their 24 face neighbours, each loaded once
  float V[2][2][2], XM[2][2], XP[2][2], YM[2][2], YP[2][2], ZM[2][2], ZP[2][2];
#pragma unroll
  for (int c = 0; c < 2; ++c)
#pragma unroll
    for (int d = 0; d < 2; ++d) {
      XM[c][d] = p[xo[0] + yo[1 + d] + zo[1 + c]];
      XP[c][d] = p[xo[3] + yo[1 + d] + zo[1 + c]];
      YM[c][d] = p[xo[1 + d] + yo[0] + zo[1 + c]];
      YP[c][d] = p[xo[1 + d] + yo[3] + zo[1 + c]];
      ZM[c][d] = p[xo[1 + d] + yo[1 + c] + zo[0]];
      ZP[c][d] = p[xo[1 + d] + yo[1 + c] + zo[3]];
#pragma unroll
      for (int a = 0; a < 2; ++a) V[c][d][a] = p[xo[1 + a] + yo[1 + d] + zo[1 + c]];
    }
  float acc = 0.f;
#pragma unroll
  for (int dz = 0; dz < 2; ++dz)
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
      for (int dx = 0; dx < 2; ++dx) {
        const int i = i0 + dx, j = j0 + dy, k = k0 + dz;
        const float xm = dx ? V[dz][dy][0] : XM[dz][dy], xp = dx ? XP[dz][dy] : V[dz][dy][1];
        const float ym = dy ? V[dz][0][dx] : YM[dz][dx], yp = dy ? YP[dz][dx] : V[dz][1][dx];
        const float zm = dz ? V[0][dy][dx] : ZM[dy][dx], zp = dz ? ZP[dy][dx] : V[1][dy][dx];
        float diag = (MASK && ball_coarse(u)) ? ball_diag(u, i, j, k)
                     : mg_simple(periodic, gam, d0) ? 6.0f
                                                    : mg_diag(i, j, k, s, periodic, gam, d0);
        float s0 = nb6(xm, xp, ym, yp, zm, zp);
        // children outside the ball solve's mask carry no residual
        if (!MASK || g_in(u, i, j, k))
          acc = __fadd_rn(acc, resid_value(s0, V[dz][dy][dx], b.base[gidx(b, i, j, k)], diag,
                                           inv_h2));
      }
  int cc = gidx(uc, I, J, K);
  bc.base[cc] = __fmul_rn(0.125f, acc);
  uc.base[cc] = 0.0f;
}

template <bool MASK>
__global__ void __launch_bounds__(256) k_resid_restrict(Grid u, Grid b, float inv_h2,
                                                        Grid uc, Grid bc, int periodic,
                                                        float gam, float d0) {
  pdl_wait();
  pdl_release();
  d_resid_restrict<MASK>(bi_native(), u, b, inv_h2, uc, bc, periodic, gam, d0);
}

// ---------------------------------------------------------------------------
// u += P uc: trilinear interpolation of the cell-centred coarse correction
// (weights 3/4 on the parent, 1/4 on the next coarse cell per axis).  Coarse
// ghosts are zero (open) or wrap (periodic).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float prolong_value(Grid uc, int i, int j, int k, int periodic,
                                               float gam_c) {
  const int sc = uc.s;
  int I = i >> 1, J = j >> 1, K = k >> 1;
  int I2 = (i & 1) ? I + 1 : I - 1;
  int J2 = (j & 1) ? J + 1 : J - 1;
  int K2 = (k & 1) ? K + 1 : K - 1;
  // open: a coarse ghost is -gam_c times the interior value beside it (per
  // axis), see bnd_diag
  float fx = 1.0f, fy = 1.0f, fz = 1.0f;
  if (periodic) {
    I2 = I2 < 0 ? sc - 1 : (I2 >= sc ? 0 : I2);
    J2 = J2 < 0 ? sc - 1 : (J2 >= sc ? 0 : J2);
    K2 = K2 < 0 ? sc - 1 : (K2 >= sc ? 0 : K2);
  } else {
    if (I2 < 0 || I2 >= sc) { I2 = I; fx = -gam_c; }
    if (J2 < 0 || J2 >= sc) { J2 = J; fy = -gam_c; }
    if (K2 < 0 || K2 >= sc) { K2 = K; fz = -gam_c; }
  }
  const float* q = uc.base;
  return prolong_mix(q[gidx(uc, I, J, K)], q[gidx(uc, I2, J, K)], q[gidx(uc, I, J2, K)],
                     q[gidx(uc, I2, J2, K)], q[gidx(uc, I, J, K2)], q[gidx(uc, I2, J, K2)],
                     q[gidx(uc, I, J2, K2)], q[gidx(uc, I2, J2, K2)], fx, fy, fz);
}

// The ball solve's prolongation value v: as prolong_value, with the masked
// coarse level's own boundary (a second coarse cell outside the mask is the
// parent times -ball_gam); false (no correction) where the parent itself is
// outside the coarse mask.
__device__ __forceinline__ bool prolong_value_ball(Grid uc, int i, int j, int k, float& v) {
  const int I = i >> 1, J = j >> 1, K = k >> 1;
  if (!g_in(uc, I, J, K)) return false;
  int I2 = (i & 1) ? I + 1 : I - 1, J2 = (j & 1) ? J + 1 : J - 1, K2 = (k & 1) ? K + 1 : K - 1;
  float fx = 1.0f, fy = 1.0f, fz = 1.0f;
  if (!g_in(uc, I2, J, K)) { fx = -ball_gam(uc, I, J, K, 0, I2 > I ? 1 : -1); I2 = I; }
  if (!g_in(uc, I, J2, K)) { fy = -ball_gam(uc, I, J, K, 1, J2 > J ? 1 : -1); J2 = J; }
  if (!g_in(uc, I, J, K2)) { fz = -ball_gam(uc, I, J, K, 2, K2 > K ? 1 : -1); K2 = K; }
  const float* q = uc.base;
  v = prolong_mix(q[gidx(uc, I, J, K)], q[gidx(uc, I2, J, K)], q[gidx(uc, I, J2, K)],
                  q[gidx(uc, I2, J2, K)], q[gidx(uc, I, J, K2)], q[gidx(uc, I2, J, K2)],
                  q[gidx(uc, I, J2, K2)], q[gidx(uc, I2, J2, K2)], fx, fy, fz);
  return true;
}

template <bool MASK>
__device__ __forceinline__ void d_prolong(const BI& bi, Grid uc, Grid u, int periodic,
                                                 float gam_c){
  const int s = u.s;
  int i = bi.x * blockDim.x + threadIdx.x;
  int j = bi.y * blockDim.y + threadIdx.y;
  int k = bi.z;
  if (i >= s || j >= s || (MASK && !g_in(u, i, j, k))) return;
  float* p = u.base + gidx(u, i, j, k);
  if (MASK && uc.mbase) {
    float v;
    if (prolong_value_ball(uc, i, j, k, v)) *p = __fadd_rn(*p, v);
    return;
  }
  *p = __fadd_rn(*p, prolong_value(uc, i, j, k, periodic, gam_c));
}

template <bool MASK>
__global__ void __launch_bounds__(256) k_prolong(Grid uc, Grid u, int periodic,
                                                 float gam_c) {
  pdl_wait();
  pdl_release();
  d_prolong<MASK>(bi_native(), uc, u, periodic, gam_c);
}

// out-of-place form: w = u + P uc (w and u may be different layouts).  One
// thread per coarse cell: its 3x3x3 coarse neighbourhood is loaded once and
// its 8 fine children take prolong_value's arithmetic on those values.
__global__ void __launch_bounds__(256) k_prolong_to(Grid uc, Grid u, Grid w, int periodic,
                                                    float gam_c) {
  pdl_wait();
  pdl_release();
  const int sc = uc.s;
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  const int K = blockIdx.z;
  if (I >= sc || J >= sc) return;
  if (uc.mbase) {  // the ball solve: its children one by one (mask of u)
#pragma unroll 1
    for (int c = 0; c < 8; ++c) {
      const int i = 2 * I + (c & 1), j = 2 * J + ((c >> 1) & 1), k = 2 * K + (c >> 2);
      float uv = u.base[gidx(u, i, j, k)], v;
      if (g_in(u, i, j, k) && prolong_value_ball(uc, i, j, k, v)) uv = __fadd_rn(uv, v);
      w.base[gidx(w, i, j, k)] = uv;
    }
    return;
  }
  // coarse index of offset o in {-1, 0, +1} along an axis: wrapped, or (open)
  // the cell itself when outside, with factor -gam_c applied below
  auto idx = [&](int c, int o) {
    int v = c + o;
    if (v < 0 || v >= sc) v = periodic ? (v < 0 ? sc - 1 : 0) : c;
    return v;
  };
  auto fac = [&](int c, int o) {
    int v = c + o;
    return (!periodic && (v < 0 || v >= sc)) ? -gam_c : 1.0f;
  };
  int xi[3], yi[3], zi[3];
  float fxv[3], fyv[3], fzv[3];
#pragma unroll
  for (int o = 0; o < 3; ++o) {
    xi[o] = idx(I, o - 1);
    yi[o] = idx(J, o - 1);
    zi[o] = idx(K, o - 1);
    fxv[o] = fac(I, o - 1);
    fyv[o] = fac(J, o - 1);
    fzv[o] = fac(K, o - 1);
  }
  float Q[3][3][3];  // [z][y][x]
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int a = 0; a < 3; ++a) Q[c][b][a] = uc.base[gidx(uc, xi[a], yi[b], zi[c])];
#pragma unroll
  for (int dz = 0; dz < 2; ++dz)
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
      for (int dx = 0; dx < 2; ++dx) {
        // the child's second coarse cell per axis: below for an even child,
        // above for an odd one (neighbourhood index 0 or 2)
        const int ax = dx ? 2 : 0, ay = dy ? 2 : 0, az = dz ? 2 : 0;
        const float fx = fxv[ax], fy = fyv[ay], fz = fzv[az];
        const float fxy = __fmul_rn(fx, fy), fxz = __fmul_rn(fx, fz), fyz = __fmul_rn(fy, fz);
        const float fxyz = __fmul_rn(fxy, fz);
        const float c000 = Q[1][1][1], c100 = __fmul_rn(fx, Q[1][1][ax]);
        const float c010 = __fmul_rn(fy, Q[1][ay][1]), c110 = __fmul_rn(fxy, Q[1][ay][ax]);
        const float c001 = __fmul_rn(fz, Q[az][1][1]), c101 = __fmul_rn(fxz, Q[az][1][ax]);
        const float c011 = __fmul_rn(fyz, Q[az][ay][1]);
        const float c111 = __fmul_rn(fxyz, Q[az][ay][ax]);
        const float a0 = lerp34(c000, c100), a1 = lerp34(c010, c110);
        const float a2 = lerp34(c001, c101), a3 = lerp34(c011, c111);
        const float pv = lerp34(lerp34(a0, a1), lerp34(a2, a3));
        const int i = 2 * I + dx, j = 2 * J + dy, k = 2 * K + dz;
        w.base[gidx(w, i, j, k)] = __fadd_rn(u.base[gidx(u, i, j, k)], pv);
      }
}


static inline dim3 grid_half(int s) {
  return dim3((unsigned)(((s / 2 + 1) / 2 + 31) / 32), (unsigned)((s + 7) / 8), (unsigned)s);
}
static inline dim3 grid_full(int s) { return dim3((unsigned)((s + 31) / 32), (unsigned)((s + 7) / 8), (unsigned)s); }

void launch_rbgs(cudaStream_t st, Grid u, Grid b, float h2, int color, int periodic,
                 float gam, int zero_start, float d0) {
  if (u.mbase)
    launch_pdl(k_rbgs<true>, grid_half(u.s), dim3(32, 8), 0, st, u, b, h2, color, periodic, gam,
               zero_start, d0);
  else
    launch_pdl(k_rbgs<false>, grid_half(u.s), dim3(32, 8), 0, st, u, b, h2, color, periodic,
               gam, zero_start, d0);
  note_launch();
}
void launch_resid_restrict(cudaStream_t st, Grid u, Grid b, float inv_h2, Grid uc, Grid bc,
                           int periodic, float gam, float d0) {
  if (u.mbase)
    launch_pdl(k_resid_restrict<true>, grid_full(uc.s), dim3(32, 8), 0, st, u, b, inv_h2, uc, bc,
               periodic, gam, d0);
  else
    launch_pdl(k_resid_restrict<false>, grid_full(uc.s), dim3(32, 8), 0, st, u, b, inv_h2, uc,
               bc, periodic, gam, d0);
  note_launch();
}
// ghost layer of src copied into d1 and d2 (same side, any layouts)
__global__ void k_copy_ghosts(Grid src, Grid d1, Grid d2) {
  const int s = src.s, n = s + 2;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < 6 * n * n;
       t += gridDim.x * blockDim.x) {
    const int f = t / (n * n), r = t - f * n * n;
    const int a = r % n - 1, c = r / n - 1, side = (f & 1) ? s : -1;
    int i, j, k;
    if (f < 2) { i = side; j = a; k = c; }
    else if (f < 4) { i = a; j = side; k = c; }
    else { i = a; j = c; k = side; }
    const float v = src.base[gidx(src, i, j, k)];
    d1.base[gidx(d1, i, j, k)] = v;
    d2.base[gidx(d2, i, j, k)] = v;
  }
}

void launch_copy_ghosts(cudaStream_t st, Grid src, Grid d1, Grid d2) {
  const int n = src.s + 2;
  int blocks = (6 * n * n + 255) / 256;
  k_copy_ghosts<<<blocks < 1024 ? blocks : 1024, 256, 0, st>>>(src, d1, d2);
  note_launch();
}

void launch_prolong_to(cudaStream_t st, Grid uc, Grid u, Grid w, int periodic, float gam_c) {
  launch_pdl(k_prolong_to, grid_full(uc.s), dim3(32, 8), 0, st, uc, u, w, periodic, gam_c);
  note_launch();
}
void launch_prolong(cudaStream_t st, Grid uc, Grid u, int periodic, float gam_c) {
  if (u.mbase)
    launch_pdl(k_prolong<true>, grid_full(u.s), dim3(32, 8), 0, st, uc, u, periodic, gam_c);
  else
    launch_pdl(k_prolong<false>, grid_full(u.s), dim3(32, 8), 0, st, uc, u, periodic, gam_c);
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
// With CORRECT the potential is first advanced by the V-cycle's correction,
// Phi' = Phi + e (the e grid has zero ghosts / the same wrap), evaluated on
// the fly at all 7 stencil points; Phi' is written out of place to (qh, ql)
// and the residual is that of Phi'.  NC: the grids are read through the
// non-coherent cache (they do not change during the launch); the persistent
// solve, which rewrites them between its phases, reads them from L2.
template <bool NC>
__device__ __forceinline__ float ldx(const float* p) {
  if (NC) return __ldg(p);
  return __ldcg(p);
}

template <bool CORRECT, bool NC = true, bool MASK = false>
__device__ __forceinline__ void d_defect(const BI& bi, Grid ph, Grid pl, Grid e, Grid qh, Grid ql,
                                                Grid fh, Grid fl, Grid rb, int periodic,
                                                int write_r, double* __restrict__ partial,
                                                unsigned int* counter, double* __restrict__ out,
                                                float d0, float d0l){
  const int s = ph.s;
  int i = bi.x * blockDim.x + threadIdx.x;
  int j = bi.y * blockDim.y + threadIdx.y;
  float r2 = 0.f;
  // a contiguous run of planes per thread; the (i, j) column's values at
  // k-1, k, k+1 (with the correction added) roll through registers
  const int chunk = (s + bi.gz - 1) / bi.gz;
  int k0 = bi.z * chunk, k1 = min(s, k0 + chunk);
  if (MASK && i < s && j < s) {
    // the ball solve: only the column's mask cells (outside, both potential
    // buffers hold the same boundary values, and no pass reads r there)
    int m0, m1;
    mask_column(ph, i, j, m0, m1);
    k0 = max(k0, m0);
    k1 = min(k1, m1);
  }
  if (i < s && j < s && k0 < k1) {
    const int xm = wrap_m(i, s, periodic) - i, xp = wrap_p(i, s, periodic) - i;
    const int ym = wrap_m(j, s, periodic) - j, yp = wrap_p(j, s, periodic) - j;
    // the column's raw values at plane kk (hi, lo and, with CORRECT, e),
    // then the corrected double-float value of Phi from them
    float cH, cL, cE = 0.0f;
    auto column_load = [&](int kk) {
      const int c = gidx(ph, i, j, kk);
      cH = ldx<NC>(ph.base + c);
      cL = ldx<NC>(pl.base + c);
      if (CORRECT) cE = ldx<NC>(e.base + gidx(e, i, j, kk));
    };
    auto column_value = [&](float& H, float& L) {
      H = cH;
      L = cL;
      if (CORRECT) {
        df t = two_sum(H, cE);
        H = t.hi;
        L = __fadd_rn(L, t.lo);
      }
    };
    float Hm, Lm, Hc, Lc, Hp, Lp;
    column_load(wrap_m(k0, s, periodic));
    column_value(Hm, Lm);
    column_load(k0);
    column_value(Hc, Lc);
    // the column at k + 1 (the z+ neighbour of plane k) is loaded one plane
    // ahead of its use: in the iteration of plane k - 1 (k0 - 1: here)
    column_load(wrap_p(k0, s, periodic));
    const int off[4] = {xm, xp, ym * ph.sy, yp * ph.sy};
    const int eoff[4] = {xm, xp, ym * e.sy, yp * e.sy};
    // the in-plane neighbours (with their corrections) and f of plane k are
    // loaded one iteration ahead, so their latency overlaps the arithmetic
    // of the plane before (none of them is written by this kernel)
    float nh[4], nl[4], ne[4], nfh, nfl;
    auto load_plane = [&](int k) {
      const int c = gidx(ph, i, j, k);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        nh[q] = ldx<NC>(ph.base + c + off[q]);
        nl[q] = ldx<NC>(pl.base + c + off[q]);
        if (CORRECT) ne[q] = ldx<NC>(e.base + gidx(e, i, j, k) + eoff[q]);
      }
      const int fc = gidx(fh, i, j, k);
      nfh = ldx<NC>(fh.base + fc);
      nfl = ldx<NC>(fl.base + fc);
    };
    load_plane(k0);
    for (int k = k0; k < k1; ++k) {
      float H[7], Lo[7], E[4];
      H[0] = Hc;
      Lo[0] = Lc;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        H[q + 1] = nh[q];
        Lo[q + 1] = nl[q];
        E[q] = ne[q];
      }
      float sacc = nfh;
      float comp = nfl;
      column_value(Hp, Lp);
      if (k + 1 < k1) {
        column_load(wrap_p(k + 1, s, periodic));  // plane k + 2 <= k1 <= s
        load_plane(k + 1);
      }
      H[5] = Hm;
      Lo[5] = Lm;
      H[6] = Hp;
      Lo[6] = Lp;
      if (CORRECT) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          df t = two_sum(H[q + 1], E[q]);
          H[q + 1] = t.hi;
          Lo[q + 1] = __fadd_rn(Lo[q + 1], t.lo);
        }
        df n = fast_two_sum(H[0], Lo[0]);
        int qc = gidx(qh, i, j, k);
        qh.base[qc] = n.hi;
        ql.base[qc] = n.lo;
      }
      // r = f - sum_nb + 6 phi: TwoSum cascade on the hi parts, rounding errors
      // and lo parts in a float compensation term
      df t;
#pragma unroll
      for (int q = 1; q < 7; ++q) {
        t = two_sum(sacc, -H[q]);
        sacc = t.hi;
        comp += t.lo;
      }
      df p6 = two_prod(d0, H[0]);
      p6.lo = __fmaf_rn(d0l, H[0], p6.lo);  // d0 = d0 + d0l exactly (diffusion shift)
      t = two_sum(sacc, p6.hi); sacc = t.hi; comp += t.lo + p6.lo;
      comp -= (Lo[1] + Lo[2]) + (Lo[3] + Lo[4]) + (Lo[5] + Lo[6]);
      comp += d0 * Lo[0];
      float r = sacc + comp;
      if (write_r) rb.base[gidx(rb, i, j, k)] = r;
      r2 = __fmaf_rn(r, r, r2);
      Hm = Hc; Lm = Lc; Hc = Hp; Lc = Lp;
    }
  }
  __shared__ double sm[32];
  float vf = warp_sumf_all(r2);
  int lane = (threadIdx.y * blockDim.x + threadIdx.x) & 31;
  int warp = (threadIdx.y * blockDim.x + threadIdx.x) >> 5;
  if (lane == 0) sm[warp] = (double)vf;
  __syncthreads();
  unsigned nblk = bi.gx * bi.gy * bi.gz;
  unsigned bid = bi.x + bi.gx * (bi.y + bi.gy * bi.z);
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

template <bool CORRECT, bool MASK>
__global__ void __launch_bounds__(256) k_defect(Grid ph, Grid pl, Grid e, Grid qh, Grid ql,
                                                Grid fh, Grid fl, Grid rb, int periodic,
                                                int write_r, double* __restrict__ partial,
                                                unsigned int* counter, double* __restrict__ out,
                                                float d0, float d0l) {
  pdl_wait();
  pdl_release();
  d_defect<CORRECT, true, MASK>(bi_native(), ph, pl, e, qh, ql, fh, fl, rb, periodic, write_r,
                                partial, counter, out, d0, d0l);
}

static inline dim3 grid_defect(int s) {
  return dim3((unsigned)((s + 31) / 32), (unsigned)((s + 7) / 8), (unsigned)(s < 16 ? s : 16));
}
int defect_blocks(int s) {
  dim3 g = grid_defect(s);
  return (int)(g.x * g.y * g.z);
}

void launch_defect(cudaStream_t st, Grid ph, Grid pl, const Grid* e, Grid qh, Grid ql,
                   Grid fh, Grid fl, Grid rb, int periodic, bool write_r, double* partial,
                   unsigned int* counter, double* out, double d0) {
  const float d0h = (float)d0, d0l = (float)(d0 - (double)d0h);
  const int w = write_r ? 1 : 0;
  const dim3 g = grid_defect(ph.s), blk(32, 8);
  if (e && ph.mbase)
    launch_pdl(k_defect<true, true>, g, blk, 0, st, ph, pl, *e, qh, ql, fh, fl, rb, periodic, w,
               partial, counter, out, d0h, d0l);
  else if (e)
    launch_pdl(k_defect<true, false>, g, blk, 0, st, ph, pl, *e, qh, ql, fh, fl, rb, periodic, w,
               partial, counter, out, d0h, d0l);
  else if (ph.mbase)
    launch_pdl(k_defect<false, true>, g, blk, 0, st, ph, pl, ph, qh, ql, fh, fl, rb, periodic, w,
               partial, counter, out, d0h, d0l);
  else
    launch_pdl(k_defect<false, false>, g, blk, 0, st, ph, pl, ph, qh, ql, fh, fl, rb, periodic, w,
               partial, counter, out, d0h, d0l);
  note_launch();
}

// Phi (hi, lo) += e.
__global__ void __launch_bounds__(256) k_correct(Grid ph, Grid pl, Grid e) {
  pdl_wait();
  pdl_release();
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
  launch_pdl(k_correct, grid_full(ph.s), dim3(32, 8), 0, st, ph, pl, e);
  note_launch();
}

// Dense [z][y][x] FP32 arrays of side s <-> grid interiors (the learned
// guess and training-pair capture).  to_dense: d (=|+=) g; from_dense:
// g (=|+=) d.
__global__ void __launch_bounds__(256) k_to_dense(Grid g, float* __restrict__ d, int add) {
  const int s = g.s;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  int k = blockIdx.z;
  if (i >= s || j >= s) return;
  long long o = ((long long)k * s + j) * s + i;
  float v = g.base[gidx(g, i, j, k)];
  d[o] = add ? d[o] + v : v;
}

__global__ void __launch_bounds__(256) k_from_dense(const float* __restrict__ d, Grid g, int add) {
  const int s = g.s;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  int k = blockIdx.z;
  if (i >= s || j >= s) return;
  long long o = ((long long)k * s + j) * s + i;
  int c = gidx(g, i, j, k);
  g.base[c] = add ? g.base[c] + d[o] : d[o];
}

void launch_to_dense(cudaStream_t st, Grid g, float* d, bool add) {
  k_to_dense<<<grid_full(g.s), dim3(32, 8), 0, st>>>(g, d, add ? 1 : 0);
  note_launch();
}
void launch_from_dense(cudaStream_t st, const float* d, Grid g, bool add) {
  k_from_dense<<<grid_full(g.s), dim3(32, 8), 0, st>>>(d, g, add ? 1 : 0);
  note_launch();
}

// Warm start extrapolated in time: Phi <- Phi + w (Phi - Phi_prev),
// Phi_prev <- old Phi (interior only; the ghost layer keeps its boundary
// values).  Double-float when `pair`, FP32 hi only otherwise.
__device__ __forceinline__ void d_predict(const BI& bi, Grid ph, Grid pl, Grid qh, Grid ql, float w,
                                                 int pair){
  const int s = ph.s;
  int i = bi.x * blockDim.x + threadIdx.x;
  int j = bi.y * blockDim.y + threadIdx.y;
  int k = bi.z;
  if (i >= s || j >= s) return;
  int c = gidx(ph, i, j, k);
  if (pair) {
    df cur{ph.base[c], pl.base[c]}, prev{qh.base[c], ql.base[c]};
    df d = df_add(cur, df{-prev.hi, -prev.lo});
    df v = df_add(cur, df_mul(d, df{w, 0.0f}));
    qh.base[c] = cur.hi;
    ql.base[c] = cur.lo;
    ph.base[c] = v.hi;
    pl.base[c] = v.lo;
  } else {
    float cur = ph.base[c], prev = qh.base[c];
    qh.base[c] = cur;
    ph.base[c] = cur + w * (cur - prev);
  }
}

__global__ void __launch_bounds__(256) k_predict(Grid ph, Grid pl, Grid qh, Grid ql, float w,
                                                 int pair) {
  pdl_wait();
  pdl_release();
  d_predict(bi_native(), ph, pl, qh, ql, w, pair);
}

void launch_predict(cudaStream_t st, Grid ph, Grid pl, Grid qh, Grid ql, float w, bool pair) {
  launch_pdl(k_predict, grid_full(ph.s), dim3(32, 8), 0, st, ph, pl, qh, ql, w, pair ? 1 : 0);
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

// ---------------------------------------------------------------------------
// Batched forms (one launch over the member realisations of a table).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) kb_rbgs(const RbgsDesc* d, const BTable* t,
                                               const int* active) {
  int q;
  BI bi;
  if (!batch_map(d, t, active, q, bi)) return;
  const RbgsDesc& e = d[q];
  each_plane(bi, e.u.s, [&](const BI& b) {
    d_rbgs<false>(b, e.u, e.b, e.h2, e.color, e.periodic, e.gam, e.zero_start, 6.0f);
  });
}
__global__ void __launch_bounds__(256) kb_restrict(const RestrictDesc* d, const BTable* t,
                                                   const int* active) {
  int q;
  BI bi;
  if (!batch_map(d, t, active, q, bi)) return;
  const RestrictDesc& e = d[q];
  each_plane(bi, e.uc.s, [&](const BI& b) {
    d_resid_restrict<false>(b, e.u, e.b, e.inv_h2, e.uc, e.bc, e.periodic, e.gam, 6.0f);
  });
}
__global__ void __launch_bounds__(256) kb_prolong(const ProlongDesc* d, const BTable* t,
                                                  const int* active) {
  int q;
  BI bi;
  if (!batch_map(d, t, active, q, bi)) return;
  const ProlongDesc& e = d[q];
  each_plane(bi, e.u.s,
             [&](const BI& b) { d_prolong<false>(b, e.uc, e.u, e.periodic, e.gam_c); });
}
__global__ void __launch_bounds__(256, 4) kb_defect(const DefectDesc* d, const BTable* t,
                                                 const int* active) {
  int q;
  BI bi;
  if (!batch_map(d, t, active, q, bi)) return;
  const DefectDesc& e = d[q];
  if (e.iters) {
    const int k = e.iters[e.r];
    if (k == 0)
      d_defect<false>(bi, e.ph, e.pl, e.e, e.ph, e.pl, e.fh, e.fl, e.rb, e.periodic, e.write_r,
                      e.partial, e.counter, e.out, 6.0f, 0.0f);
    else if (((k - 1) & 1) == 0)
      d_defect<true>(bi, e.ph, e.pl, e.e, e.qh, e.ql, e.fh, e.fl, e.rb, e.periodic, e.write_r,
                     e.partial, e.counter, e.out, 6.0f, 0.0f);
    else
      d_defect<true>(bi, e.qh, e.ql, e.e, e.ph, e.pl, e.fh, e.fl, e.rb, e.periodic, e.write_r,
                     e.partial, e.counter, e.out, 6.0f, 0.0f);
    return;
  }
  if (e.correct)
    d_defect<true>(bi, e.ph, e.pl, e.e, e.qh, e.ql, e.fh, e.fl, e.rb, e.periodic, e.write_r,
                   e.partial, e.counter, e.out, 6.0f, 0.0f);
  else
    d_defect<false>(bi, e.ph, e.pl, e.e, e.qh, e.ql, e.fh, e.fl, e.rb, e.periodic, e.write_r,
                    e.partial, e.counter, e.out, 6.0f, 0.0f);
}
__global__ void kb_solve_init(int R, int* active, int* iters, int* failed) {
  const int r = (int)threadIdx.x;
  if (r < R) {
    active[r] = 1;
    iters[r] = 0;
    failed[r] = 0;
  }
}
__global__ void kb_converged(int R, const double* __restrict__ scal,
                             const double* __restrict__ rtol, const int* __restrict__ maxv,
                             int* active, int* iters, int* failed, double* rel,
                             cudaGraphConditionalHandle loop) {
  const int r = (int)threadIdx.x;
  int on = 0;
  if (r < R && active[r]) {
    const double f2 = scal[16 * r], r2 = scal[16 * r + 11];
    const double v = f2 > 0.0 ? sqrt(r2 / f2) : 0.0;
    rel[r] = v;
    if (v <= rtol[r] || f2 == 0.0) {
      active[r] = 0;
    } else if (iters[r] >= maxv[r]) {
      active[r] = 0;
      failed[r] = 1;
    } else {
      iters[r] += 1;
      on = 1;
    }
  }
  const int any = __syncthreads_or(on);
  if (r == 0) cudaGraphSetConditional(loop, any ? 1u : 0u);
}
void launch_solve_init_b(cudaStream_t st, int R, int* active, int* iters, int* failed) {
  kb_solve_init<<<1, MAX_REAL, 0, st>>>(R, active, iters, failed);
  note_launch();
}
void launch_converged_b(cudaStream_t st, int R, const double* scal, const double* rtol,
                        const int* maxv, int* active, int* iters, int* failed, double* rel,
                        cudaGraphConditionalHandle loop) {
  kb_converged<<<1, MAX_REAL, 0, st>>>(R, scal, rtol, maxv, active, iters, failed, rel, loop);
  note_launch();
}
__global__ void __launch_bounds__(256) kb_predict(const PredictDesc* d, const BTable* t) {
  int q;
  BI bi;
  if (!batch_map(d, t, (const int*)nullptr, q, bi)) return;
  const PredictDesc& e = d[q];
  each_plane(bi, e.ph.s, [&](const BI& b) { d_predict(b, e.ph, e.pl, e.qh, e.ql, e.w, e.pair); });
}

void launch_rbgs_b(cudaStream_t st, int grid, const RbgsDesc* d, const BTable* t,
                   const int* active, int bx, int by) {
  if (grid <= 0) return;
  kb_rbgs<<<grid, dim3(bx, by), 0, st>>>(d, t, active);
  note_launch();
}
void launch_restrict_b(cudaStream_t st, int grid, const RestrictDesc* d, const BTable* t,
                       const int* active) {
  if (grid <= 0) return;
  kb_restrict<<<grid, dim3(32, 8), 0, st>>>(d, t, active);
  note_launch();
}
void launch_prolong_b(cudaStream_t st, int grid, const ProlongDesc* d, const BTable* t,
                      const int* active) {
  if (grid <= 0) return;
  kb_prolong<<<grid, dim3(32, 8), 0, st>>>(d, t, active);
  note_launch();
}
void launch_defect_b(cudaStream_t st, int grid, const DefectDesc* d, const BTable* t,
                     const int* active) {
  if (grid <= 0) return;
  kb_defect<<<grid, dim3(32, 8), 0, st>>>(d, t, active);
  note_launch();
}
void launch_predict_b(cudaStream_t st, int grid, const PredictDesc* d, const BTable* t) {
  if (grid <= 0) return;
  kb_predict<<<grid, dim3(32, 8), 0, st>>>(d, t);
  note_launch();
}

// the grid of a batched pass over s planes: BZ planes per block
static inline dim3 zchunk(dim3 g) { return dim3(g.x, g.y, (g.z + BZ - 1) / BZ); }

dim3 rbgs_grid(int s) { return grid_half(s); }
// the colour pass with bx x by blocks: each thread takes two cells of its
// colour in a row, so a row needs ceil(s/4) threads
dim3 rbgs_grid(int s, int bx, int by) {
  const int tx = ((s >> 1) + 1) / 2;
  return dim3((unsigned)((tx + bx - 1) / bx), (unsigned)((s + by - 1) / by), (unsigned)s);
}
dim3 full_grid(int s) { return grid_full(s); }
dim3 defect_grid(int s) { return grid_defect(s); }
dim3 rbgs_grid_b(int s, int bx, int by) { return zchunk(rbgs_grid(s, bx, by)); }
dim3 full_grid_b(int s) { return zchunk(grid_full(s)); }

// ---------------------------------------------------------------------------
// Persistent batched solve.  One cooperative launch (all blocks resident)
// takes every realisation of a batch from its starting potential to its
// tolerance: defect (with the V-cycle's correction applied), the
// convergence test, and the V-cycle's passes, each pass over all still
// active realisations, separated by a grid-wide barrier.  The decisions are
// those of a single context's host loop (Sec. 2.1 solve; stop once
// ||f - A Phi|| / ||f|| <= rtol), taken by every block alike from the same
// residual norms, so no host read happens inside a solve.
// ---------------------------------------------------------------------------
namespace {

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned atom_add_acq_rel_u32(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;"
               : "=r"(old)
               : "l"(p), "r"(v)
               : "memory");
  return old;
}
__device__ __forceinline__ int ld_volatile_i32(const int* p) {
  return *(const volatile int*)p;
}

// Grid-wide barrier with a bounded wait.  Thread 0 of each block reads the
// generation, arrives, and either (last arrival) resets the count and
// publishes the next generation, or polls the generation until it changes,
// the barrier's error word is set, or limit_ns has passed (then it sets the
// error word and the phase).  Returns false, in every thread of the block,
// once the barrier has failed: the caller leaves the kernel.
__device__ bool grid_barrier(GridBar* g, unsigned expected, unsigned long long limit_ns,
                             int phase) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    int good = ld_volatile_i32(&g->err) == 0;
    if (good) {
      __threadfence();
      const unsigned gen = ld_acquire_u32(&g->gen);
      const unsigned arrived = atom_add_acq_rel_u32(&g->count, 1u) + 1u;
      if (arrived == expected) {
        g->count = 0u;
        st_release_u32(&g->gen, gen + 1u);
      } else {
        const unsigned long long t0 = global_ns();
        while (ld_acquire_u32(&g->gen) == gen) {
          if (ld_volatile_i32(&g->err)) {
            good = 0;
            break;
          }
          if (global_ns() - t0 > limit_ns) {
            if (atomicCAS(&g->err, 0, 1) == 0) atomicExch(&g->where, phase);
            good = 0;
            break;
          }
          __nanosleep(100);
        }
      }
      __threadfence();
    }
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

constexpr int SOLVE_NT = 256;  // 32 x 8 threads: the block of every batched mesh pass

// The blocks of table t, taken by the blocks of the grid in turn: block
// blockIdx.x takes blocks blockIdx.x, blockIdx.x + gridDim.x, ...  The table's
// block offsets are staged in shared memory (s_off, MAX_MEMBERS + 1 ints) and
// the member is found by walking forward (members are in block order), so a
// block costs no dependent global loads beyond its descriptor; the blocks of
// inactive realisations are skipped member by member.
template <class D, class F>
__device__ __forceinline__ void each_block(const D* d, const BTable* t, const int* act,
                                           int* s_off, F&& f) {
  const int tid = (int)(threadIdx.x + threadIdx.y * blockDim.x);
  __syncthreads();  // the previous phase's readers of s_off are done
  const int m = t->m;
  for (int i = tid; i <= m; i += (int)(blockDim.x * blockDim.y)) s_off[i] = t->off[i];
  __syncthreads();
  if (m <= 0) return;
  const int tot = s_off[m], G = (int)gridDim.x;
  int q = 0;
  int b = (int)blockIdx.x;
  while (b < tot) {
    while (s_off[q + 1] <= b) ++q;
    const D& e = d[q];
    if (act && !act[e.r]) {
      // the first block of this grid block's sequence past member q
      const int next = s_off[q + 1];
      b = next + ((((int)blockIdx.x - next) % G) + G) % G;
      continue;
    }
    const int lb = b - s_off[q];
    const BI bi{lb % e.gx, (lb / e.gx) % e.gy, lb / (e.gx * e.gy), e.gx, e.gy, e.gz};
    f(e, bi);
    __syncthreads();  // the passes' shared reduction words are reused
    b += G;
  }
}

template <int MINB>
__global__ void __launch_bounds__(SOLVE_NT, MINB) kb_solve(SolveArgs a) {
  extern __shared__ float cc_sm[];
  __shared__ int act[MAX_REAL], it[MAX_REAL];
  __shared__ float red[CC_NT / 32];
  __shared__ CcLevel lev[CC_MAXL];
  __shared__ int nlev;
  __shared__ int s_off[MAX_MEMBERS + 1];
  const int tid = (int)(threadIdx.x + threadIdx.y * blockDim.x);
  const unsigned expected = gridDim.x + (unsigned)a.extra;
  for (int r = tid; r < a.R; r += SOLVE_NT) {
    act[r] = 1;
    it[r] = 0;
  }
  __syncthreads();
  int phase = 0;
  for (;;) {
    // defect: after V-cycle k >= 1 the correction e moves the potential from
    // the buffer of parity k - 1 into that of parity k (k = 0: no correction)
    each_block(a.def, a.def_t, act, s_off, [&](const DefectDesc& e, const BI& bi) {
      const int k = it[e.r];
      if (k == 0)
        d_defect<false, false>(bi, e.ph, e.pl, e.e, e.ph, e.pl, e.fh, e.fl, e.rb, e.periodic,
                               e.write_r, e.partial, e.counter, e.out, 6.0f, 0.0f);
      else if (((k - 1) & 1) == 0)
        d_defect<true, false>(bi, e.ph, e.pl, e.e, e.qh, e.ql, e.fh, e.fl, e.rb, e.periodic,
                              e.write_r, e.partial, e.counter, e.out, 6.0f, 0.0f);
      else
        d_defect<true, false>(bi, e.qh, e.ql, e.e, e.ph, e.pl, e.fh, e.fl, e.rb, e.periodic,
                              e.write_r, e.partial, e.counter, e.out, 6.0f, 0.0f);
    });
    if (!grid_barrier(a.bar, expected, a.limit_ns, phase++)) return;
    // convergence test of every active realisation, the same in every block
    if (tid < a.R && act[tid]) {
      const int r = tid;
      const double f2 = __ldcg(a.scal + 16 * r), r2 = __ldcg(a.scal + 16 * r + 11);
      const double v = f2 > 0.0 ? sqrt(r2 / f2) : 0.0;
      if (blockIdx.x == 0) a.rel[r] = v;
      if (v <= a.rtol[r] || f2 == 0.0) {
        act[r] = 0;
      } else if (it[r] >= a.maxv[r]) {
        act[r] = 0;
        if (blockIdx.x == 0) a.failed[r] = 1;
      } else {
        it[r] += 1;
      }
    }
    if (!__syncthreads_or(tid < a.R && act[tid])) break;
    // one V(2,2) cycle of every active realisation, pass by pass
    for (int sl = 0; sl < a.n_slots; ++sl) {
      const SolveSlot S = a.slots[sl];
      if (S.kind == SLOT_RBGS) {
        each_block((const RbgsDesc*)S.d, S.t, act, s_off,
                   [&](const RbgsDesc& e, const BI& bi) {
                     each_plane(bi, e.u.s, [&](const BI& b) {
                       d_rbgs<false>(b, e.u, e.b, e.h2, e.color, e.periodic, e.gam,
                                     e.zero_start, 6.0f);
                     });
                   });
      } else if (S.kind == SLOT_RESTRICT) {
        each_block((const RestrictDesc*)S.d, S.t, act, s_off,
                   [&](const RestrictDesc& e, const BI& bi) {
                     each_plane(bi, e.uc.s, [&](const BI& b) {
                       d_resid_restrict<false>(b, e.u, e.b, e.inv_h2, e.uc, e.bc, e.periodic, e.gam,
                                        6.0f);
                     });
                   });
      } else if (S.kind == SLOT_PROLONG) {
        each_block((const ProlongDesc*)S.d, S.t, act, s_off,
                   [&](const ProlongDesc& e, const BI& bi) {
                     each_plane(bi, e.u.s,
                                [&](const BI& b) {
                                  d_prolong<false>(b, e.uc, e.u, e.periodic, e.gam_c);
                                });
                   });
      } else {  // SLOT_CMG: the coarse levels of one realisation per block
        const CmgDesc* cd = (const CmgDesc*)S.d;
        for (int q = (int)blockIdx.x; q < S.n; q += (int)gridDim.x) {
          const CmgDesc& e = cd[q];
          if (!act[e.r]) continue;
          if (a.fast_coarse && fc_supported(e.u.s)) {
            fc_vcycle<SOLVE_NT, false>(cc_sm, red, e.u, e.b, e.level, e.periodic, e.sweeps,
                                       e.zero_top, 0.0f);
            continue;
          }
          if (tid == 0) Cc<1, SOLVE_NT>::init_levels(lev, nlev, e.u.s, e.level, e.periodic, 0.0f);
          __syncthreads();
          Cc<1, SOLVE_NT> c;
          c.sm = cc_sm;
          c.my = 0;
          c.periodic = e.periodic;
          c.sweeps = e.sweeps;
          c.nlev = nlev;
          c.sig0 = 0.0f;
          c.gu = e.u;
          c.gb = e.b;
          c.V = lev;
          c.init_pointers(lev);
          __syncthreads();
          c.run(e.zero_top, red);
          __syncthreads();
        }
      }
      if (!grid_barrier(a.bar, expected, a.limit_ns, phase++)) return;
    }
  }
  if (blockIdx.x == 0)
    for (int r = tid; r < a.R; r += SOLVE_NT) a.iters[r] = it[r];
  // the gradient field of each final potential (in the start buffer after an
  // even number of V-cycles, in the other one after an odd number)
  each_block(a.grad, a.grad_t, (const int*)nullptr, s_off, [&](const GradDesc& e, const BI& bi) {
    const bool odd = (it[e.r] & 1) != 0;
    d_grad(bi, odd ? e.ph_alt : e.ph, odd ? e.pl_alt : e.pl, e.n, e.lo, e.s, e.periodic, e.G);
  });
}

int solve_smem() { return cmg_smem_bytes(cmg_top_side(1)); }

// blocks per SM the kernel is compiled for: 4 by default (64 registers,
// small spills; measured 14.2 ms per batch48 step), 2 with PM_SOLVE_MINB=2
// (no spill, half the occupancy; 15.4 ms)
int solve_minb() {
  const char* v = getenv("PM_SOLVE_MINB");
  return v && atoi(v) == 2 ? 2 : 4;
}

template <int MINB>
int solve_grid_t() {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaFuncSetAttribute(kb_solve<MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           solve_smem()) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kb_solve<MINB>, SOLVE_NT,
                                                    solve_smem()) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return per * sms;
}

}  // namespace

int solve_grid_b() {
  static int grid = -1;
  if (grid < 0) grid = solve_minb() == 4 ? solve_grid_t<4>() : solve_grid_t<2>();
  return grid;
}

cudaError_t launch_solve_b(cudaStream_t st, const SolveArgs& a) {
  const int grid = solve_grid_b();
  if (grid <= 0) return cudaErrorLaunchOutOfResources;
  SolveArgs arg = a;
  void* params[] = {(void*)&arg};
  const void* fn = solve_minb() == 4 ? (const void*)kb_solve<4> : (const void*)kb_solve<2>;
  cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(32, 8), params,
                                              (size_t)solve_smem(), st);
  note_launch();
  return e;
}

}  // namespace pm
