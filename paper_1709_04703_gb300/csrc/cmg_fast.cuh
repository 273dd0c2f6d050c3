// The coarse levels of the multigrid V-cycle (Sec. 2.1, Eq. 3) in one CTA,
// for tops of side <= 16 (16, 14, 12, 10, 8, 7, 6, 5, 4, 3, 2): the sides are template
// constants, so every index is plain constant arithmetic, and each level's
// unknowns carry a one-cell halo in shared memory that holds the open
// boundary's ghost values (the Dirichlet data on the top level, zero below
// it), so only the periodic wrap needs a branch; with the ball solve's mask
// (the top Grid's mask fields) only the mask's cells are updated, with the
// masked coarse boundaries of pm_common.cuh.  The operations and their
// order are those of the per-level kernels and of the generic form
// (cmg_dev.cuh), through the same arithmetic (mg_arith.cuh): the results are
// the same bits.
#pragma once
#include "mg_arith.cuh"
#include "pm_kernels.cuh"

namespace pm {

namespace {

// the next coarser side (0 at the bottom: side <= 4 or odd), as in cc_layout
__host__ __device__ constexpr int fc_next(int S) { return (S <= 4 || (S & 1)) ? 0 : S / 2; }
// shared floats of the levels from side S down: u padded (S+2)^3, b S^3
__host__ __device__ constexpr int fc_floats(int S) {
  return (S + 2) * (S + 2) * (S + 2) + S * S * S + (fc_next(S) ? fc_floats(fc_next(S)) : 0);
}
// the largest top the fast form takes
constexpr int FC_MAX_TOP = 16;
__host__ __device__ inline bool fc_supported(int S) {
  return S == 16 || S == 14 || S == 12 || S == 10 || S == 8 || S == 7 || S == 6 || S == 5 ||
         S == 4 || S == 3 || S == 2;
}

template <int S>
__device__ __forceinline__ int fc_p(int i, int j, int k) {
  return ((k + 1) * (S + 2) + (j + 1)) * (S + 2) + (i + 1);
}
template <int S>
__device__ __forceinline__ int fc_d(int i, int j, int k) {
  return (k * S + j) * S + i;
}

// Level constants, computed as the generic form computes them
struct FcLev {
  float h2, inv_h2, gam, d0;
  bool simple;
};

// MASK: the ball solve's masked levels (compiled out of the unmasked form)
template <int NT, bool MASK>
struct Fc {
  int periodic, sweeps, lev0;
  float sig0;
  Grid gu, gb;  // the top level in global memory (its ghost layer: the Dirichlet data)

  // the ball solve's mask of level q (side S): the top's mask fields with
  // the step doubling per level; only its cells are updated, and a coarse
  // level's boundary is ball_gam's
  __device__ Grid lvl(int q, int S) const {
    Grid g = gu;
    g.mstep = gu.mstep << q;
    g.s = S;
    return g;
  }
  template <int S>
  __device__ bool in(int q, int i, int j, int k) const {
    return !MASK || g_in(lvl(q, S), i, j, k);
  }

  __device__ static int lt() { return (int)(threadIdx.x + threadIdx.y * blockDim.x); }

  __device__ FcLev lev(int q) const {
    FcLev v;
    const float H = (float)(1 << (lev0 + q));
    v.h2 = H * H;
    v.inv_h2 = 1.0f / v.h2;
    v.gam = MASK ? 0.0f : (H - 1.0f) / (H + 1.0f);
    v.d0 = 6.0f + sig0 * v.h2;
    v.simple = mg_simple(periodic, v.gam, v.d0);
    return v;
  }

  // the six neighbours of cell (i, j, k) (padded index p) summed as nb6 does
  template <int S>
  __device__ __forceinline__ float nbs(const float* u, int i, int j, int k, int p) const {
    constexpr int P = S + 2, P2 = P * P;
    int xm = p - 1, xp = p + 1, ym = p - P, yp = p + P, zm = p - P2, zp = p + P2;
    if (periodic) {
      if (i == 0) xm += S;
      if (i == S - 1) xp -= S;
      if (j == 0) ym += S * P;
      if (j == S - 1) yp -= S * P;
      if (k == 0) zm += S * P2;
      if (k == S - 1) zp -= S * P2;
    }
    return nb6(u[xm], u[xp], u[ym], u[yp], u[zm], u[zp]);
  }

  template <int S>
  __device__ __forceinline__ float diag(const FcLev& L, int i, int j, int k, int q) const {
    if (MASK && (gu.mstep << q) > 2) return ball_diag(lvl(q, S), i, j, k);
    return L.simple ? 6.0f : mg_diag(i, j, k, S, periodic, L.gam, L.d0);
  }
  // the Gauss-Seidel value's form: exact x(1/6) only without a coarse mask
  __device__ bool simple(const FcLev& L, int q) const {
    return L.simple && !(MASK && (gu.mstep << q) > 2);
  }

  // one colour of red-black SOR (sor_value) on an even level, two cells per
  // thread at a time (loads of both before either store: cells of one
  // colour never neighbour each other)
  template <int S>
  __device__ void smooth(float* u, const float* b, const FcLev& L, int colour, int q) const {
    constexpr int H = S / 2, N = S * S * H;
    auto cell = [&](int t, int& i, int& j, int& k) {
      const int r = t / H;
      j = r % S;
      k = r / S;
      i = 2 * (t % H) + ((j + k + colour) & 1);
    };
    for (int a = lt(); a < N; a += 2 * NT) {
      const int c2 = a + NT;
      int i1, j1, k1, i2 = 0, j2 = 0, k2 = 0;
      cell(a, i1, j1, k1);
      const int p1 = fc_p<S>(i1, j1, k1);
      const float s1 = nbs<S>(u, i1, j1, k1, p1);
      const float b1 = b[fc_d<S>(i1, j1, k1)];
      float s2 = 0.0f, b2 = 0.0f;
      int p2 = 0;
      if (c2 < N) {
        cell(c2, i2, j2, k2);
        p2 = fc_p<S>(i2, j2, k2);
        s2 = nbs<S>(u, i2, j2, k2, p2);
        b2 = b[fc_d<S>(i2, j2, k2)];
      }
      const bool sp = simple(L, q);
      // (the iterate is zeroed in shared memory before a level's first
      // sweep, so the old values are always stored ones)
      const float o1 = u[p1], o2 = c2 < N ? u[p2] : 0.0f;
      if (in<S>(q, i1, j1, k1))
        u[p1] = sor_value(o1, gs_value(s1, b1, L.h2, sp, diag<S>(L, i1, j1, k1, q)));
      if (c2 < N && in<S>(q, i2, j2, k2))
        u[p2] = sor_value(o2, gs_value(s2, b2, L.h2, sp, diag<S>(L, i2, j2, k2, q)));
    }
  }

  // coarse b = 1/8 of the sum over the 8 children of the fine residual; the
  // coarse u is zeroed
  template <int S>
  __device__ void restrict_to(const float* u, const float* b, const FcLev& L, float* uc,
                              float* bc, int q) const {
    constexpr int C = S / 2, N = C * C * C;
    for (int t = lt(); t < N; t += NT) {
      const int I = t % C, J = (t / C) % C, K = t / (C * C);
      float acc = 0.0f;
#pragma unroll
      for (int dz = 0; dz < 2; ++dz)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
          for (int dx = 0; dx < 2; ++dx) {
            const int i = 2 * I + dx, j = 2 * J + dy, k = 2 * K + dz;
            if (!in<S>(q, i, j, k)) continue;  // no residual outside the mask
            const int p = fc_p<S>(i, j, k);
            const float s0 = nbs<S>(u, i, j, k, p);
            acc = __fadd_rn(acc, resid_value(s0, u[p], b[fc_d<S>(i, j, k)],
                                             diag<S>(L, i, j, k, q), L.inv_h2));
          }
      bc[fc_d<C>(I, J, K)] = __fmul_rn(0.125f, acc);
      uc[fc_p<C>(I, J, K)] = 0.0f;
    }
  }

  // u += the trilinear prolongation of the coarse level (gc: its gam)
  template <int S>
  __device__ void prolong_from(float* u, const float* uc, float gc, int q) const {
    constexpr int C = S / 2, N = S * S * S;
    for (int t = lt(); t < N; t += NT) {
      const int i = t % S, j = (t / S) % S, k = t / (S * S);
      if (!in<S>(q, i, j, k)) continue;
      const int I = i >> 1, J = j >> 1, K = k >> 1;
      int I2 = (i & 1) ? I + 1 : I - 1, J2 = (j & 1) ? J + 1 : J - 1;
      int K2 = (k & 1) ? K + 1 : K - 1;
      float fx = 1.0f, fy = 1.0f, fz = 1.0f;
      if (MASK) {
        // the masked coarse level's own boundary; no correction where the
        // parent is outside its mask
        const Grid cg = lvl(q + 1, C);
        if (!g_in(cg, I, J, K)) continue;
        if (!g_in(cg, I2, J, K)) { fx = -ball_gam(cg, I, J, K, 0, I2 > I ? 1 : -1); I2 = I; }
        if (!g_in(cg, I, J2, K)) { fy = -ball_gam(cg, I, J, K, 1, J2 > J ? 1 : -1); J2 = J; }
        if (!g_in(cg, I, J, K2)) { fz = -ball_gam(cg, I, J, K, 2, K2 > K ? 1 : -1); K2 = K; }
      } else if (periodic) {
        I2 = I2 < 0 ? C - 1 : (I2 >= C ? 0 : I2);
        J2 = J2 < 0 ? C - 1 : (J2 >= C ? 0 : J2);
        K2 = K2 < 0 ? C - 1 : (K2 >= C ? 0 : K2);
      } else {
        if (I2 < 0 || I2 >= C) { I2 = I; fx = -gc; }
        if (J2 < 0 || J2 >= C) { J2 = J; fy = -gc; }
        if (K2 < 0 || K2 >= C) { K2 = K; fz = -gc; }
      }
      const float pv = prolong_mix(uc[fc_p<C>(I, J, K)], uc[fc_p<C>(I2, J, K)],
                                   uc[fc_p<C>(I, J2, K)], uc[fc_p<C>(I2, J2, K)],
                                   uc[fc_p<C>(I, J, K2)], uc[fc_p<C>(I2, J, K2)],
                                   uc[fc_p<C>(I, J2, K2)], uc[fc_p<C>(I2, J2, K2)], fx, fy, fz);
      const int p = fc_p<S>(i, j, k);
      u[p] = __fadd_rn(u[p], pv);
    }
  }

  // mean over the S^3 cells of u (padded) or b, in the generic form's fixed
  // order: CC_NT virtual threads, virtual thread t summing cells t, t + CC_NT,
  // ...; warp sums; the CC_NT / 32 warps in order (red: CC_NT / 32 floats)
  template <int S>
  __device__ float mean(const float* v, bool padded, float* red) const {
    static_assert(CC_NT % NT == 0, "the block size divides CC_NT");
    constexpr int N = S * S * S;
    __syncthreads();
#pragma unroll
    for (int rep = 0; rep < CC_NT / NT; ++rep) {
      const int vt = lt() + rep * NT;
      float acc = 0.0f;
      for (int t = vt; t < N; t += CC_NT)
        acc += padded ? v[fc_p<S>(t % S, (t / S) % S, t / (S * S))] : v[t];
      acc = warp_sumf_all(acc);
      if ((vt & 31) == 0) red[vt >> 5] = acc;
    }
    __syncthreads();
    float m = 0.0f;
    for (int w = 0; w < CC_NT / 32; ++w) m += red[w];
    __syncthreads();
    return m / (float)N;
  }

  // the bottom (side <= 4 or odd): periodic Poisson has its means projected
  // out (b before, u after); Dirichlet bottoms take red-black SOR with
  // factor 2 / (1 + sin(pi / (S + 1))); periodic ones Gauss-Seidel
  // (lexicographic in one thread on an odd side)
  template <int S>
  __device__ void bottom(float* u, float* b, const FcLev& L, float* red, int q) const {
    constexpr int N = S * S * S;
    const bool proj = periodic && sig0 == 0.0f;
    if (proj) {
      const float m = mean<S>(b, false, red);
      for (int t = lt(); t < N; t += NT) b[t] -= m;
      __syncthreads();
    }
    // the side enters sinf as a run-time value, as in the generic form (a
    // constant argument could be folded by the compiler with other rounding)
    int s1 = S + 1;
    asm volatile("" : "+r"(s1));
    const float omega = periodic ? 1.0f : 2.0f / (1.0f + sinf(3.14159265f / (float)s1));
    const bool sp = simple(L, q);
    auto cell = [&](int t) {
      const int i = t % S, j = (t / S) % S, k = t / (S * S);
      if (!in<S>(q, i, j, k)) return;
      const int p = fc_p<S>(i, j, k);
      const float old = u[p];
      const float gs = gs_value(nbs<S>(u, i, j, k, p), b[t], L.h2, sp, diag<S>(L, i, j, k, q));
      u[p] = omega == 1.0f ? gs : __fmaf_rn(omega, __fsub_rn(gs, old), old);
    };
    for (int w = 0; w < sweeps; ++w) {
      if ((S & 1) && periodic) {
        if (lt() == 0)
          for (int t = 0; t < N; ++t) cell(t);
        __syncthreads();
      } else {
        for (int colour = 0; colour < 2; ++colour) {
          for (int t = lt(); t < N; t += NT) {
            const int i = t % S, j = (t / S) % S, k = t / (S * S);
            if (((i + j + k) & 1) == colour) cell(t);
          }
          __syncthreads();
        }
      }
    }
    if (proj) {
      const float m = mean<S>(u, true, red);
      for (int t = lt(); t < N; t += NT) {
        const int p = fc_p<S>(t % S, (t / S) % S, t / (S * S));
        u[p] -= m;
      }
      __syncthreads();
    }
  }

  // the V(2,2) cycle from level q (side S, shared floats at sm) down
  template <int S>
  __device__ void cycle(float* sm, int q, float* red) const {
    constexpr int P = S + 2;
    float* u = sm;
    float* b = sm + P * P * P;
    const FcLev L = lev(q);
    if constexpr (fc_next(S) == 0) {
      bottom<S>(u, b, L, red, q);
      __syncthreads();
    } else {
      constexpr int C = S / 2;
      float* uc = b + S * S * S;
      float* bc = uc + (C + 2) * (C + 2) * (C + 2);
      for (int p = 0; p < 4; ++p) {
        smooth<S>(u, b, L, p & 1, q);
        __syncthreads();
      }
      restrict_to<S>(u, b, L, uc, bc, q);
      __syncthreads();
      cycle<C>(uc, q + 1, red);
      prolong_from<S>(u, uc, lev(q + 1).gam, q);
      __syncthreads();
      for (int p = 0; p < 4; ++p) {
        smooth<S>(u, b, L, p & 1, q);
        __syncthreads();
      }
    }
  }

  // halos of the levels from side S down: the top's (q == 0) open-boundary
  // faces from the ghost layer of gu, everything else zero
  template <int S>
  __device__ void halos(float* sm, int q) const {
    constexpr int P = S + 2, N = P * P * P;
    for (int t = lt(); t < N; t += NT) {
      const int i = t % P - 1, j = (t / P) % P - 1, k = t / (P * P) - 1;
      const int out = (i < 0 || i >= S) + (j < 0 || j >= S) + (k < 0 || k >= S);
      if (out == 0) continue;
      sm[t] = (q == 0 && !periodic && out == 1) ? gu.base[gidx(gu, i, j, k)] : 0.0f;
    }
    if constexpr (fc_next(S) != 0) halos<fc_next(S)>(sm + P * P * P + S * S * S, q + 1);
  }

  // the whole V-cycle from a top of side S: load, cycle, store
  template <int S>
  __device__ void run(float* sm, int zero_top, float* red) const {
    constexpr int P = S + 2, N = S * S * S;
    halos<S>(sm, 0);
    float* u = sm;
    float* b = sm + P * P * P;
    for (int t = lt(); t < N; t += NT) {
      const int i = t % S, j = (t / S) % S, k = t / (S * S);
      b[t] = gb.base[gidx(gb, i, j, k)];
      u[fc_p<S>(i, j, k)] = zero_top ? 0.0f : gu.base[gidx(gu, i, j, k)];
    }
    __syncthreads();
    cycle<S>(sm, 0, red);
    for (int t = lt(); t < N; t += NT) {
      const int i = t % S, j = (t / S) % S, k = t / (S * S);
      gu.base[gidx(gu, i, j, k)] = u[fc_p<S>(i, j, k)];
    }
    __syncthreads();
  }
};

// the V-cycle from a top of side S0 (fc_supported(S0)) in one CTA of NT
// threads; sm holds fc_floats(FC_MAX_TOP) floats, red CC_NT / 32
template <int NT, bool MASK>
__device__ void fc_vcycle(float* sm, float* red, Grid u, Grid b, int level, int periodic,
                          int sweeps, int zero_top, float sig0) {
  Fc<NT, MASK> f;
  f.periodic = periodic;
  f.sweeps = sweeps;
  f.lev0 = level;
  f.sig0 = sig0;
  f.gu = u;
  f.gb = b;
  switch (u.s) {
    case 16: f.template run<16>(sm, zero_top, red); break;
    case 14: f.template run<14>(sm, zero_top, red); break;
    case 12: f.template run<12>(sm, zero_top, red); break;
    case 10: f.template run<10>(sm, zero_top, red); break;
    case 8: f.template run<8>(sm, zero_top, red); break;
    case 7: f.template run<7>(sm, zero_top, red); break;
    case 6: f.template run<6>(sm, zero_top, red); break;
    case 5: f.template run<5>(sm, zero_top, red); break;
    case 4: f.template run<4>(sm, zero_top, red); break;
    case 3: f.template run<3>(sm, zero_top, red); break;
    case 2: f.template run<2>(sm, zero_top, red); break;
    default: break;  // not reached: callers check fc_supported
  }
}

}  // namespace

}  // namespace pm
