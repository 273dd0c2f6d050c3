// The update arithmetic of the multigrid smoother and transfers (Sec. 2.1,
// Eq. 3 as the 7-point system on level l, spacing h_l = 2^l in cells),
// shared by every kernel that applies it: the one-colour passes, the fused
// two-sweep pass, the batched forms and the cluster-resident coarse levels.
// Written with explicit round-to-nearest operations so that all of them
// produce the same bits.
#pragma once

#include "pm_common.cuh"

namespace pm {

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
// Diagonal with a shift: the operator sum_nb u - d0 u (d0 = 6 + sig h^2 for
// the implicit diffusion substeps, 6 for Poisson) plus the coarse open
// ghost term.  "simple" (d0 = 6, no ghost term) keeps the exact x(1/6) form.
__device__ __forceinline__ float mg_diag(int i, int j, int k, int s, int periodic, float gam,
                                         float d0) {
  if (periodic) return d0;
  int nb = (i == 0) + (i == s - 1) + (j == 0) + (j == s - 1) + (k == 0) + (k == s - 1);
  return d0 + gam * (float)nb;
}
__device__ __forceinline__ bool mg_simple(int periodic, float gam, float d0) {
  return (periodic || gam == 0.0f) && d0 == 6.0f;
}

// The update arithmetic of the smoother and the transfers, written with
// explicit round-to-nearest operations so that every kernel that applies
// them (one colour per launch, the fused two-sweep pass, the batched forms)
// produces the same bits.
__device__ __forceinline__ float nb6(float xm, float xp, float ym, float yp, float zm, float zp) {
  return __fadd_rn(__fadd_rn(__fadd_rn(xm, xp), __fadd_rn(ym, yp)), __fadd_rn(zm, zp));
}
// Gauss-Seidel value (sum_nb u - h^2 b) / diag
__device__ __forceinline__ float gs_value(float s0, float bv, float h2, bool simple, float diag) {
  float t = __fsub_rn(s0, __fmul_rn(h2, bv));
  return simple ? __fmul_rn(t, 1.0f / 6.0f) : __fdiv_rn(t, diag);
}
// Red-black SOR (MG_OMEGA, pm_common.cuh): a smoothing update moves the cell
// from its old value towards the Gauss-Seidel value by MG_OMEGA; every
// smoothing pass of every FP32 form applies it, so they all keep giving the
// same bits.  A zero old value may be read or assumed: the result is the
// same.
__device__ __forceinline__ float sor_value(float old, float gs) {
  return MG_OMEGA == 1.0f ? gs : __fmaf_rn(MG_OMEGA, __fsub_rn(gs, old), old);
}
// residual b - (sum_nb u - diag u) / h^2
__device__ __forceinline__ float resid_value(float s0, float uc, float bv, float diag,
                                             float inv_h2) {
  float lap = __fsub_rn(s0, __fmul_rn(diag, uc));
  return __fsub_rn(bv, __fmul_rn(lap, inv_h2));
}
// trilinear weights 3/4, 1/4 per axis (x, then y, then z)
__device__ __forceinline__ float lerp34(float a, float b) {
  return __fadd_rn(__fmul_rn(0.75f, a), __fmul_rn(0.25f, b));
}

// The trilinear prolongation value of a fine child from its coarse parent
// q000 and the next coarse cells per axis (q100 along x, q010 along y, ...;
// q110 the xy-diagonal one and so on), with the open-boundary factors fx,
// fy, fz (1, or -gam_c where the next coarse cell is a ghost)
__device__ __forceinline__ float prolong_mix(float q000, float q100, float q010, float q110,
                                             float q001, float q101, float q011, float q111,
                                             float fx, float fy, float fz) {
  const float fxy = __fmul_rn(fx, fy), fxz = __fmul_rn(fx, fz), fyz = __fmul_rn(fy, fz);
  const float fxyz = __fmul_rn(fxy, fz);
  const float c100 = __fmul_rn(fx, q100), c010 = __fmul_rn(fy, q010);
  const float c110 = __fmul_rn(fxy, q110), c001 = __fmul_rn(fz, q001);
  const float c101 = __fmul_rn(fxz, q101), c011 = __fmul_rn(fyz, q011);
  const float c111 = __fmul_rn(fxyz, q111);
  const float a0 = lerp34(q000, c100), a1 = lerp34(c010, c110);
  const float a2 = lerp34(c001, c101), a3 = lerp34(c011, c111);
  return lerp34(lerp34(a0, a1), lerp34(a2, a3));
}

// Centred difference of the double-float potential (hi + lo pairs) between
// mesh points p and m: (hp - hm) + (lp - lm), as the gather's force uses it.
__device__ __forceinline__ float gdiff(float hp, float hm, float lp, float lm) {
  return __fadd_rn(__fsub_rn(hp, hm), __fsub_rn(lp, lm));
}

// The gradient field of the potential at cell (i, j, k) of the active cube
// (lo, side s) on the padded (n + 2)^3 mesh: G = the centred differences
// along x, y, z (wrapped when periodic), one float4 per cell.
__device__ __forceinline__ void d_grad(const BI& bi, const float* ph, const float* pl, int n,
                                       int lo, int s, int periodic, float4* G) {
  const int P = n + 2;
  const int i = bi.x * blockDim.x + threadIdx.x, j = bi.y * blockDim.y + threadIdx.y;
  const int k = bi.z;
  if (i >= s || j >= s) return;
  const int X = lo + i, Y = lo + j, Z = lo + k;
  auto w = [&](int a) { return periodic ? (a < 0 ? a + n : (a >= n ? a - n : a)) : a; };
  const long long c = ((long long)(Z + 1) * P + (Y + 1)) * P + (X + 1);
  const long long xm = ((long long)(Z + 1) * P + (Y + 1)) * P + (w(X - 1) + 1);
  const long long xp = ((long long)(Z + 1) * P + (Y + 1)) * P + (w(X + 1) + 1);
  const long long ym = ((long long)(Z + 1) * P + (w(Y - 1) + 1)) * P + (X + 1);
  const long long yp = ((long long)(Z + 1) * P + (w(Y + 1) + 1)) * P + (X + 1);
  const long long zm = ((long long)(w(Z - 1) + 1) * P + (Y + 1)) * P + (X + 1);
  const long long zp = ((long long)(w(Z + 1) + 1) * P + (Y + 1)) * P + (X + 1);
  G[c] = make_float4(gdiff(ph[xp], ph[xm], pl[xp], pl[xm]), gdiff(ph[yp], ph[ym], pl[yp], pl[ym]),
                     gdiff(ph[zp], ph[zm], pl[zp], pl[zm]), 0.0f);
}

}  // namespace pm
