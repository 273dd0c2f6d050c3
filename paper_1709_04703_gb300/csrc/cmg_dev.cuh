// The coarse levels of the multigrid V-cycle (Sec. 2.1, Eq. 3 on levels of
// side <= 64) solved inside one CTA or one thread-block cluster: the level
// layout in shared memory, the per-level constants, and the smoothing,
// restriction, prolongation and bottom passes.  Used by the coarse-level
// kernels (k_cmg.cu) and by the persistent batched solve (k_mg.cu).
#pragma once
#include <cooperative_groups.h>

#include "mg_arith.cuh"
#include "pm_kernels.cuh"

namespace pm {

namespace cg = cooperative_groups;

namespace {

constexpr int CC_NT = 512;   // threads per CTA (16 warps: 128 registers each)
constexpr int CC_NY = CC_NT / 32;  // rows of a plane taken at once (one warp per row)
constexpr int CC_MAXL = 8;   // levels of a cluster V-cycle

// Layout of the levels of a cluster V-cycle from top side S0 in each CTA's
// shared memory, identical in every CTA so that a cell has the same offset
// wherever it lives.  Level q has side S[q] (halving while even and > 4),
// np[q] planes per CTA, u at off[q] and b at off[q] + np[q] S[q]^2 floats.  A
// level of side >= CL is split over the CL CTAs by z planes (CTA r owns
// planes [floor(r S / CL), floor((r + 1) S / CL))); a smaller one lives whole
// in CTA 0.
struct CcLayout {
  int n;
  int S[CC_MAXL], np[CC_MAXL], off[CC_MAXL];
  int floats;
};

__host__ __device__ inline CcLayout cc_layout(int S0, int CL) {
  CcLayout L{};
  int S = S0, acc = 0;
  for (int q = 0; q < CC_MAXL; ++q) {
    L.S[q] = S;
    L.np[q] = S >= CL ? (S + CL - 1) / CL : S;
    L.off[q] = acc;
    acc += 2 * L.np[q] * S * S;
    L.n = q + 1;
    if (S <= 4 || (S & 1)) break;
    S /= 2;
  }
  L.floats = acc;
  return L;
}

// Per-level constants of a cluster V-cycle, in shared memory: side, planes
// per CTA, offset, the level's h^2, 1/h^2, coarse open-boundary factor and
// diagonal, the first plane of every CTA (z0[r], z0[CL] = S), the owner of
// every plane, and this CTA's pointers to every plane of u (up[k + 1] for k
// in [-1, S]: wrapped when periodic, NULL outside an open cube) and of b
// (bp[k]) in the shared memory of the CTA that holds it.
struct CcLevel {
  int S, np, off, simple;
  float h2, inv_h2, gam, d0;
  float inv_S, inv_h;  // 1/S and 2/S for the index arithmetic
  int z0[17];
  unsigned char owner[64];
  float* up[66];
  float* bp[64];
};

// q = x / d, r = x % d for 0 <= x < 2^22, 1 <= d <= 64, from a float
// reciprocal (its error is below one, so one correction step suffices)
__device__ __forceinline__ void fdivmod(int x, int d, float inv_d, int& q, int& r) {
  q = (int)((float)x * inv_d);
  r = x - q * d;
  if (r < 0) { --q; r += d; }
  else if (r >= d) { ++q; r -= d; }
}

template <int CL, int NT = CC_NT>
struct Cc {
  // linear thread index (the persistent batched solve runs 32 x 8 blocks)
  __device__ static int lt() { return (int)(threadIdx.x + threadIdx.y * blockDim.x); }
  float* sm;
  int my;             // rank of this CTA in the cluster
  int periodic, sweeps, nlev;
  float sig0;
  Grid gu, gb;        // the top level in global memory (its ghost layer: Dirichlet data)
  const CcLevel* V;   // nlev levels, in shared memory

  // the level table: constants by thread 0, then the plane pointers by all
  // threads (the caller synchronises after each part)
  __device__ static void init_levels(CcLevel* V, int& nlev, int S0, int lev0, int periodic,
                                     float sig0) {
    const CcLayout L = cc_layout(S0, CL);
    nlev = L.n;
    for (int q = 0; q < L.n; ++q) {
      CcLevel& v = V[q];
      v.S = L.S[q];
      v.np = L.np[q];
      v.off = L.off[q];
      const float H = (float)(1 << (lev0 + q));
      v.h2 = H * H;
      v.inv_h2 = 1.0f / v.h2;
      v.gam = (H - 1.0f) / (H + 1.0f);
      v.d0 = 6.0f + sig0 * v.h2;
      v.simple = mg_simple(periodic, v.gam, v.d0) ? 1 : 0;
      v.inv_S = 1.0f / (float)v.S;
      v.inv_h = 2.0f / (float)v.S;
      const bool dist = CL == 1 || v.S >= CL;
      for (int r = 0; r <= CL; ++r) v.z0[r] = dist ? (r * v.S) / CL : (r == 0 ? 0 : v.S);
      for (int k = 0; k < v.S; ++k) {
        int r = 0;
        while (v.z0[r + 1] <= k) ++r;
        v.owner[k] = (unsigned char)r;
      }
    }
  }
  __device__ void init_pointers(CcLevel* W) const {
    for (int t = lt(); t < nlev * 130; t += NT) {
      const int q = t / 130, e = t % 130;
      CcLevel& v = W[q];
      const int S = v.S;
      if (e < 66) {
        int k = e - 1;
        if (k > S) continue;
        if (k < 0 || k >= S) {
          if (!periodic) { v.up[e] = nullptr; continue; }
          k = k < 0 ? S - 1 : 0;
        }
        v.up[e] = plane(q, 0, k);
      } else {
        const int k = e - 66;
        if (k < S) v.bp[k] = plane(q, 1, k);
      }
    }
  }

  __device__ bool dist(int q) const { return CL == 1 || V[q].S >= CL; }
  __device__ int z0(int q) const { return V[q].z0[my]; }
  __device__ int z1(int q) const { return V[q].z0[my + 1]; }

  // plane k (0 <= k < S) of u (which = 0) or b (1) of level q, in the shared
  // memory of the CTA that owns it
  __device__ float* plane(int q, int which, int k) const {
    const CcLevel& v = V[q];
    const int r = v.owner[k];
    float* p = sm + v.off + (which * v.np + (k - v.z0[r])) * v.S * v.S;
    if (CL == 1 || r == my) return p;
    return cg::this_cluster().map_shared_rank(p, (unsigned)r);
  }
  // u outside an open cube: the top level's ghost layer, zero below the top
  // (coarse open ghosts are folded into the diagonal)
  __device__ float ghost(int q, int i, int j, int k) const {
    return q == 0 ? gu.base[gidx(gu, i, j, k)] : 0.0f;
  }
  // u at (i, j) of plane k, pk = V[q].up[k + 1]; i, j in [-1, S]
  __device__ float uat(int q, const float* pk, int i, int j, int k) const {
    const int S = V[q].S;
    if (periodic) {
      i = i < 0 ? S - 1 : (i >= S ? 0 : i);
      j = j < 0 ? S - 1 : (j >= S ? 0 : j);
    } else if (!pk || i < 0 || j < 0 || i >= S || j >= S) {
      return ghost(q, i, j, k);
    }
    return pk[j * S + i];
  }

  __device__ void sync(int q) const {
    if (CL == 1) {
      __syncthreads();
    } else if (dist(q)) {
      cg::this_cluster().sync();
    } else if (my == 0) {
      __syncthreads();
    }
  }
  __device__ void sync_all() const {
    if (CL == 1) __syncthreads(); else cg::this_cluster().sync();
  }

  // the six neighbours of cell (i, j) of plane k of level q, summed as nb6
  // does: pu its u plane, pm / pp the planes below and above
  __device__ float nbsum(int q, int i, int j, int k, const float* pu, const float* pm,
                         const float* pp) const {
    const int S = V[q].S, c = j * S + i;
    float xm, xp, ym, yp;
    if (i > 0 && i < S - 1) { xm = pu[c - 1]; xp = pu[c + 1]; }
    else { xm = uat(q, pu, i - 1, j, k); xp = uat(q, pu, i + 1, j, k); }
    if (j > 0 && j < S - 1) { ym = pu[c - S]; yp = pu[c + S]; }
    else { ym = uat(q, pu, i, j - 1, k); yp = uat(q, pu, i, j + 1, k); }
    const float zm = pm ? pm[c] : ghost(q, i, j, k - 1);
    const float zp = pp ? pp[c] : ghost(q, i, j, k + 1);
    return nb6(xm, xp, ym, yp, zm, zp);
  }
  // the Gauss-Seidel (or over-relaxed) value of cell (i, j, k) from its
  // neighbour sum s0, right-hand side bv and current value old
  __device__ float gsv(int q, int i, int j, int k, float s0, float bv, float old,
                       float omega) const {
    const CcLevel& v = V[q];
    const bool simple = v.simple != 0;
    const float gs = gs_value(s0, bv, v.h2, simple,
                              simple ? 6.0f : mg_diag(i, j, k, v.S, periodic, v.gam, v.d0));
    return omega == 1.0f ? gs : __fmaf_rn(omega, __fsub_rn(gs, old), old);
  }

  // cell idx of colour `colour` among this CTA's cells of an even level
  __device__ void colour_cell(int q, int idx, int colour, int& i, int& j, int& k) const {
    const CcLevel& v = V[q];
    int m, rest, kl;
    fdivmod(idx, v.S >> 1, v.inv_h, rest, m);
    fdivmod(rest, v.S, v.inv_S, kl, j);
    k = v.z0[my] + kl;
    i = 2 * m + ((j + k + colour) & 1);
  }

  // one colour of red-black SOR on an even level: cells (i+j+k) % 2
  // == colour of this CTA's planes, two per thread at a time (their loads
  // issued before either store; cells of one colour never neighbour each
  // other)
  __device__ void smooth_pass(int q, int colour, float omega = 1.0f) const {
    const CcLevel& v = V[q];
    const int S = v.S;
    const int n = (z1(q) - z0(q)) * S * (S >> 1);
    for (int a = lt(); a < n; a += 2 * NT) {
      const int b = a + NT;
      int i1, j1, k1, i2 = 0, j2 = 0, k2 = 0;
      colour_cell(q, a, colour, i1, j1, k1);
      float* u1 = v.up[k1 + 1];
      const float s1 = nbsum(q, i1, j1, k1, u1, v.up[k1], v.up[k1 + 2]);
      const float b1 = v.bp[k1][j1 * S + i1], o1 = u1[j1 * S + i1];
      float s2 = 0.0f, b2 = 0.0f, o2 = 0.0f;
      float* u2 = nullptr;
      if (b < n) {
        colour_cell(q, b, colour, i2, j2, k2);
        u2 = v.up[k2 + 1];
        s2 = nbsum(q, i2, j2, k2, u2, v.up[k2], v.up[k2 + 2]);
        b2 = v.bp[k2][j2 * S + i2];
        o2 = u2[j2 * S + i2];
      }
      u1[j1 * S + i1] = gsv(q, i1, j1, k1, s1, b1, o1, omega);
      if (b < n) u2[j2 * S + i2] = gsv(q, i2, j2, k2, s2, b2, o2, omega);
    }
  }

  // coarse b of level q + 1 = 1/8 of the sum over the 8 children of the
  // residual b - (sum_nb u - diag u) / h^2 of level q; the coarse u is zeroed
  __device__ void restrict_to(int q) const {
    const CcLevel& v = V[q];
    const CcLevel& c = V[q + 1];
    const int S = v.S, Sc = c.S;
    const bool simple = v.simple != 0;
    const int n = (z1(q + 1) - z0(q + 1)) * Sc * Sc;
    for (int t = lt(); t < n; t += NT) {
      int I, J, Kl, rest;
      fdivmod(t, Sc, c.inv_S, rest, I);
      fdivmod(rest, Sc, c.inv_S, Kl, J);
      const int K = c.z0[my] + Kl;
      float acc = 0.0f;
#pragma unroll
      for (int dz = 0; dz < 2; ++dz)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
          for (int dx = 0; dx < 2; ++dx) {
            const int i = 2 * I + dx, j = 2 * J + dy, k = 2 * K + dz;
            const float* pc = v.up[k + 1];
            const float s0 = nb6(uat(q, pc, i - 1, j, k), uat(q, pc, i + 1, j, k),
                                 uat(q, pc, i, j - 1, k), uat(q, pc, i, j + 1, k),
                                 v.up[k] ? v.up[k][j * S + i] : ghost(q, i, j, k - 1),
                                 v.up[k + 2] ? v.up[k + 2][j * S + i] : ghost(q, i, j, k + 1));
            const float diag = simple ? 6.0f : mg_diag(i, j, k, S, periodic, v.gam, v.d0);
            acc = __fadd_rn(acc, resid_value(s0, pc[j * S + i], v.bp[k][j * S + i], diag,
                                             v.inv_h2));
          }
      c.bp[K][J * Sc + I] = __fmul_rn(0.125f, acc);
      c.up[K + 1][J * Sc + I] = 0.0f;
    }
  }

  // u of level q += the trilinear prolongation of level q + 1
  __device__ void prolong_from(int q) const {
    const CcLevel& v = V[q];
    const CcLevel& c = V[q + 1];
    const int S = v.S, Sc = c.S;
    const float gc = c.gam;
    const int n = (z1(q) - z0(q)) * S * S;
    for (int t = lt(); t < n; t += NT) {
      int i, j, kl, rest;
      fdivmod(t, S, v.inv_S, rest, i);
      fdivmod(rest, S, v.inv_S, kl, j);
      const int k = v.z0[my] + kl;
      const int I = i >> 1, J = j >> 1, K = k >> 1;
      int I2 = (i & 1) ? I + 1 : I - 1, J2 = (j & 1) ? J + 1 : J - 1;
      int K2 = (k & 1) ? K + 1 : K - 1;
      float fx = 1.0f, fy = 1.0f, fz = 1.0f;
      if (periodic) {
        I2 = I2 < 0 ? Sc - 1 : (I2 >= Sc ? 0 : I2);
        J2 = J2 < 0 ? Sc - 1 : (J2 >= Sc ? 0 : J2);
        K2 = K2 < 0 ? Sc - 1 : (K2 >= Sc ? 0 : K2);
      } else {
        if (I2 < 0 || I2 >= Sc) { I2 = I; fx = -gc; }
        if (J2 < 0 || J2 >= Sc) { J2 = J; fy = -gc; }
        if (K2 < 0 || K2 >= Sc) { K2 = K; fz = -gc; }
      }
      const float* qa = c.up[K + 1];
      const float* qb = c.up[K2 + 1];
      const float pv = prolong_mix(qa[J * Sc + I], qa[J * Sc + I2], qa[J2 * Sc + I],
                                   qa[J2 * Sc + I2], qb[J * Sc + I], qb[J * Sc + I2],
                                   qb[J2 * Sc + I], qb[J2 * Sc + I2], fx, fy, fz);
      float* pu = v.up[k + 1];
      pu[j * S + i] = __fadd_rn(pu[j * S + i], pv);
    }
  }

  // mean over the S^3 cells of u (which = 0) or b (1) of a level held whole
  // by CTA 0, in a fixed order whatever the block size: CC_NT virtual
  // threads, virtual thread t summing cells t, t + CC_NT, ...; warp sums;
  // the CC_NT / 32 warps in order (red holds CC_NT / 32 floats)
  __device__ float mean0(int q, int which, float* red) const {
    static_assert(CC_NT % NT == 0, "the block size divides CC_NT");
    const int S = V[q].S, n3 = S * S * S;
    const float* v = which ? V[q].bp[0] : V[q].up[1];
    __syncthreads();
#pragma unroll
    for (int rep = 0; rep < CC_NT / NT; ++rep) {
      const int vt = lt() + rep * NT;
      float acc = 0.0f;
      for (int t = vt; t < n3; t += CC_NT) acc += v[t];
      acc = warp_sumf_all(acc);
      if ((vt & 31) == 0) red[vt >> 5] = acc;
    }
    __syncthreads();
    float m = 0.0f;
    for (int w = 0; w < CC_NT / 32; ++w) m += red[w];
    __syncthreads();
    return m / (float)n3;
  }

  // the bottom (side <= 4 or odd), CTA 0 alone: the periodic Poisson problem
  // is singular, so the mean of b is projected out before and that of u
  // after; Dirichlet bottoms take red-black SOR with the optimal factor of
  // the S^3 Dirichlet Laplacian, 2 / (1 + sin(pi / (S + 1))); periodic ones
  // Gauss-Seidel (lexicographic in one thread on an odd side, where
  // red-black does not close over the wrap)
  __device__ void bottom(int q, float* red) const {
    if (my != 0) return;
    const CcLevel& v = V[q];
    const int S = v.S, n3 = S * S * S;
    float* u = v.up[1];
    float* b = v.bp[0];
    const bool proj = periodic && sig0 == 0.0f;
    if (proj) {
      const float m = mean0(q, 1, red);
      for (int t = lt(); t < n3; t += NT) b[t] -= m;
      __syncthreads();
    }
    const float omega = periodic ? 1.0f : 2.0f / (1.0f + sinf(3.14159265f / (float)(S + 1)));
    auto cell = [&](int t) {
      const int i = t % S, j = (t / S) % S, k = t / (S * S);
      float* pu = v.up[k + 1];
      pu[j * S + i] = gsv(q, i, j, k, nbsum(q, i, j, k, pu, v.up[k], v.up[k + 2]), b[t],
                          pu[j * S + i], omega);
    };
    for (int w = 0; w < sweeps; ++w) {
      if ((S & 1) && periodic) {
        if (lt() == 0)
          for (int t = 0; t < n3; ++t) cell(t);
        __syncthreads();
      } else {
        for (int colour = 0; colour < 2; ++colour) {
          for (int t = lt(); t < n3; t += NT) {
            const int i = t % S, j = (t / S) % S, k = t / (S * S);
            if (((i + j + k) & 1) == colour) cell(t);
          }
          __syncthreads();
        }
      }
    }
    if (proj) {
      const float m = mean0(q, 0, red);
      for (int t = lt(); t < n3; t += NT) u[t] -= m;
      __syncthreads();
    }
  }

  // the whole V(2,2) from the top level: load, cycle, store
  __device__ void run(int zero_top, float* red) const {
    const CcLevel& v = V[0];
    const int S0 = v.S;
    const int n0 = (z1(0) - z0(0)) * S0 * S0;
    for (int t = lt(); t < n0; t += NT) {
      int i, j, kl, rest;
      fdivmod(t, S0, v.inv_S, rest, i);
      fdivmod(rest, S0, v.inv_S, kl, j);
      const int k = v.z0[my] + kl;
      v.bp[k][j * S0 + i] = gb.base[gidx(gb, i, j, k)];
      v.up[k + 1][j * S0 + i] = zero_top ? 0.0f : gu.base[gidx(gu, i, j, k)];
    }
    sync_all();
    const int nb = nlev - 1;  // the bottom level
    for (int q = 0; q < nb; ++q) {
      for (int p = 0; p < 4; ++p) {
        smooth_pass(q, p & 1, MG_OMEGA);
        sync(q);
      }
      restrict_to(q);
      sync(q + 1);
    }
    bottom(nb, red);
    sync(nb);
    for (int q = nb - 1; q >= 0; --q) {
      // CTA 0's work on levels it holds alone is complete before any other
      // CTA reads them
      if (!dist(q + 1) && dist(q)) sync_all();
      prolong_from(q);
      sync(q);
      for (int p = 0; p < 4; ++p) {
        smooth_pass(q, p & 1, MG_OMEGA);
        sync(q);
      }
    }
    for (int t = lt(); t < n0; t += NT) {
      int i, j, kl, rest;
      fdivmod(t, S0, v.inv_S, rest, i);
      fdivmod(rest, S0, v.inv_S, kl, j);
      const int k = v.z0[my] + kl;
      gu.base[gidx(gu, i, j, k)] = v.up[k + 1][j * S0 + i];
    }
    // no CTA leaves while another may still read its shared memory
    sync_all();
  }
};

}  // namespace

}  // namespace pm
