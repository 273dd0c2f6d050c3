// Shared device types and helpers of libpmshrink (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pmshrink.h"

namespace pm {

// A cubic grid level: `base` points at interior cell (0,0,0); neighbours are
// at +-1 (x), +-sy (y), +-sz (z).  Cells -1 and s along each axis are the
// ghost layer (open boundaries) and always exist in memory.
//
// The ball solve's mask (mbase != 0).  Level 0 (mstep = 2): the unknowns are
// the cells whose centre lies within R_M of the ball's centre c; twice a
// centre's offset from c along an axis is the odd integer mbase + 2 i
// (mbase = 2 lo + 1 - n for the cube's origin lo on the n^3 mesh), and the
// cell is in the mask iff the three squares sum to at most mr = floor(4
// R_M^2).  Coarse level l (mstep = 2^(l+1)): the cells whose centre lies
// within R_M (mrm2 = R_M^2, fine-cell units); their boundary conditions put
// the correction's zero where the finest level has it, on the sphere of
// radius R_M + 1/2 (mrb2) or the cube's ghost plane (ball_gam).
struct Grid {
  float* base;
  int s;
  int sy;
  int sz;
  int mbase, mstep, mr;
  float mrm2, mrb2;
};

__host__ __device__ inline int gidx(const Grid& g, int i, int j, int k) {
  return i + j * g.sy + k * g.sz;
}

__host__ __device__ inline int mask_axis(int mbase, int mstep, int i) {
  const int a0 = mbase + i * mstep, a1 = a0 + mstep - 2;
  return a0 > 0 ? a0 : (a1 < 0 ? -a1 : 1);
}
// centre of cell i of a masked level along an axis, fine-cell units from c
__host__ __device__ inline float mask_centre(const Grid& g, int i) {
  return 0.5f * (float)(g.mbase + i * g.mstep + (g.mstep >> 1) - 1);
}
// cell (i, j, k) is an unknown: always without a mask; outside the level's
// cube never
__host__ __device__ inline bool g_in(const Grid& g, int i, int j, int k) {
  if (g.mbase == 0) return true;
  if (i < 0 || j < 0 || k < 0 || i >= g.s || j >= g.s || k >= g.s) return false;
  if (g.mstep == 2) {
    const int x = mask_axis(g.mbase, 2, i), y = mask_axis(g.mbase, 2, j);
    const int z = mask_axis(g.mbase, 2, k);
    return x * x + y * y + z * z <= g.mr;
  }
  const float x = mask_centre(g, i), y = mask_centre(g, j), z = mask_centre(g, k);
  return x * x + y * y + z * z <= g.mrm2;
}
// Coarse ghost factor of mask cell (i, j, k) toward its neighbour along
// `axis` (0 x, 1 y, 2 z) on side sgn (+-1) when that neighbour is outside the
// mask: the ghost holds -gam times the cell's value, so that the linear
// profile through the cell centre vanishes at distance t, where the finest
// level's boundary lies (the sphere of radius R_M + 1/2, or the cube's ghost
// plane): gam = H / t - 1 for spacing H, at least 0.  On a cube face without
// a ball this is the cube's (H - 1) / (H + 1).
__host__ __device__ inline float ball_gam(const Grid& g, int i, int j, int k, int axis, int sgn) {
  const float H = (float)(g.mstep >> 1);
  const float cx = mask_centre(g, i), cy = mask_centre(g, j), cz = mask_centre(g, k);
  const float ca = axis == 0 ? cx : (axis == 1 ? cy : cz);
  const float o1 = axis == 0 ? cy : cx, o2 = axis == 2 ? cy : cz;
  const float ts = sqrtf(fmaxf(g.mrb2 - o1 * o1 - o2 * o2, 0.0f)) - (float)sgn * ca;
  const float lo_plane = 0.5f * (float)(g.mbase - 2);
  const float hi_plane = 0.5f * (float)(g.mbase + 2 * g.s * (g.mstep >> 1));
  const float tc = sgn > 0 ? hi_plane - ca : ca - lo_plane;
  const float t = fminf(ts, tc);
  return t > 0.0f ? fmaxf(H / t - 1.0f, 0.0f) : 0.0f;
}
// the diagonal of a coarse mask cell: 6 plus the ghost factors of its
// neighbours outside the mask
__host__ __device__ inline float ball_diag(const Grid& g, int i, int j, int k) {
  // a cell more than one spacing inside the ball has its neighbours inside
  {
    const float H = (float)(g.mstep >> 1);
    const float x = mask_centre(g, i), y = mask_centre(g, j), z = mask_centre(g, k);
    const float rin = sqrtf(g.mrm2) - H;
    const float lo_plane = 0.5f * (float)(g.mbase - 2);
    const float hi_plane = 0.5f * (float)(g.mbase + 2 * g.s * (g.mstep >> 1));
    if (rin > 0.0f && x * x + y * y + z * z < rin * rin && fminf(fminf(x, y), z) - H > lo_plane &&
        fmaxf(fmaxf(x, y), z) + H < hi_plane)
      return 6.0f;
  }
  float d = 6.0f;
  if (!g_in(g, i - 1, j, k)) d += ball_gam(g, i, j, k, 0, -1);
  if (!g_in(g, i + 1, j, k)) d += ball_gam(g, i, j, k, 0, 1);
  if (!g_in(g, i, j - 1, k)) d += ball_gam(g, i, j, k, 1, -1);
  if (!g_in(g, i, j + 1, k)) d += ball_gam(g, i, j, k, 1, 1);
  if (!g_in(g, i, j, k - 1)) d += ball_gam(g, i, j, k, 2, -1);
  if (!g_in(g, i, j, k + 1)) d += ball_gam(g, i, j, k, 2, 1);
  return d;
}
// The planes [k0, k1) of column (i, j) of a masked level-0 grid that hold
// mask cells (k0 >= k1: none): |mbase + 2 k| <= A, A the largest odd
// integer whose square is at most mr minus the column's x and y squares.
__host__ __device__ inline void mask_column(const Grid& g, int i, int j, int& k0, int& k1) {
  const int x = mask_axis(g.mbase, 2, i), y = mask_axis(g.mbase, 2, j);
  const int rem = g.mr - x * x - y * y;
  if (rem < 1) {
    k0 = 0;
    k1 = 0;
    return;
  }
  int A = (int)sqrtf((float)rem);
  while (A * A > rem) --A;
  while ((A + 1) * (A + 1) <= rem) ++A;
  if (!(A & 1)) --A;  // offsets are odd
  // mbase + 2 k in [-A, A]; mbase and A are odd, so both ends are exact
  k0 = (-A - g.mbase) / 2;
  k1 = (A - g.mbase) / 2 + 1;
}
// a masked coarse level (its cells' diagonal is ball_diag)
__host__ __device__ inline bool ball_coarse(const Grid& g) { return g.mbase != 0 && g.mstep > 2; }

// The same view of a double grid (the FP64 solve)
struct GridD {
  double* base;
  int s;
  int sy;
  int sz;
};

// Block coordinates of one launch: the native blockIdx / gridDim, or those of
// a realisation's share of a batched launch.
struct BI {
  int x, y, z, gx, gy, gz;
};
__device__ __forceinline__ BI bi_native() {
  return BI{(int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z,
            (int)gridDim.x, (int)gridDim.y, (int)gridDim.z};
}

// Programmatic dependent launch (the V-cycle's kernels): a kernel launched
// with that attribute may be scheduled while its predecessor in the stream
// still runs, so it waits for the predecessor's completion (and memory)
// before its first memory access, then lets its own successor be scheduled.
// Both are no-ops in a kernel launched normally.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Neighbour index along one axis: wraps when periodic, else may reach the
// ghost at -1 / s.
__device__ __forceinline__ int wrap_m(int i, int s, int periodic) {
  return (i == 0 && periodic) ? s - 1 : i - 1;
}
__device__ __forceinline__ int wrap_p(int i, int s, int periodic) {
  return (i == s - 1 && periodic) ? 0 : i + 1;
}

// ---------------------------------------------------------------------------
// double-float arithmetic: value = hi + lo, |lo| <= ulp(hi)/2.  Error-free
// transforms of Knuth (TwoSum) and Dekker (FastTwoSum, TwoProd via FMA),
// written with round-to-nearest intrinsics so that no contraction changes
// them.
// ---------------------------------------------------------------------------
struct df {
  float hi, lo;
};

__device__ __forceinline__ df two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ df fast_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return {s, e};
}
__device__ __forceinline__ df two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  float e = __fmaf_rn(a, b, -p);
  return {p, e};
}
__device__ __forceinline__ df df_add(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  df t = two_sum(a.lo, b.lo);
  s.lo = __fadd_rn(s.lo, t.hi);
  s = fast_two_sum(s.hi, s.lo);
  s.lo = __fadd_rn(s.lo, t.lo);
  return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df df_mul(df a, df b) {
  df p = two_prod(a.hi, b.hi);
  p.lo = __fadd_rn(p.lo, __fadd_rn(__fmul_rn(a.hi, b.lo), __fmul_rn(a.lo, b.hi)));
  return fast_two_sum(p.hi, p.lo);
}

// Keep test of the lightcone shrink: the cube klo <= x_d <= khi (exact
// float bounds of max_d |x_d - c| <= R), or with on = 1 the ball
// ((x - c)^2 + (y - c)^2) + (z - c)^2 <= r2 in FP64 (each square exact).
struct KeepBall {
  int on;
  double c, r2;
};
__device__ __forceinline__ bool in_keep(const float4& x, float klo, float khi,
                                        const KeepBall& kb) {
  if (kb.on) {
    const double dx = (double)x.x - kb.c, dy = (double)x.y - kb.c, dz = (double)x.z - kb.c;
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)) <=
           kb.r2;
  }
  return x.x >= klo && x.x <= khi && x.y >= klo && x.y <= khi && x.z >= klo && x.z <= khi;
}

// Non-negative 64-bit count -> (hi, lo) float pair, without 64-bit
// conversions (those run on the FP64 pipe, 1/64 rate on GB300): v is split
// into three 24-bit digits, each exact in float, and summed error-free.
// Exact for v < 2^72 up to the final rounding of lo (relative 2^-48).
__device__ __forceinline__ df df_from_u64(unsigned long long v) {
  float a = (float)(unsigned)(v >> 48) * 281474976710656.0f;            // 2^48
  float b = (float)(unsigned)((v >> 24) & 0xffffffu) * 16777216.0f;      // 2^24
  float c = (float)(unsigned)(v & 0xffffffu);
  df s = two_sum(a, b);
  df t = two_sum(s.hi, c);
  return fast_two_sum(t.hi, __fadd_rn(s.lo, t.lo));
}

__device__ __forceinline__ float warp_sumf_all(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------
// Fixed-point CIC node and weight along one axis (exact for any float u):
//   iq = floor(u * 2^16) - 2^15 = floor((u - 1/2) * 2^16),
//   i  = iq >> 16 (floor division),  dq = iq & 0xffff.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cic_axis(float u, int& i, int& dq) {
  int iq = __float2int_rd(__fmul_rn(u, 65536.0f)) - 32768;
  i = iq >> 16;
  dq = iq & 0xffff;
}

// Warp-level sum of a double (all lanes get it).
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sumf(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide reduction of NV doubles into out[NV] (thread 0 holds result).
template <int NV>
__device__ inline void block_sum(double (&v)[NV], double* smem /* 32*NV */) {
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    double w = warp_sum(v[q]);
    if (lane == 0) smem[warp * NV + q] = w;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double w = lane < nw ? smem[lane * NV + q] : 0.0;
      v[q] = warp_sum(w);
    }
  }
  __syncthreads();
}

}  // namespace pm

namespace pm {

// The multigrid smoother's over-relaxation factor (red-black SOR; 1 would
// be Gauss-Seidel).  Over-relaxation speeds up the V-cycle's smoothing of
// the 7-point operator: on a cell-centred periodic model of this V(2,2)
// cycle (the same transfers) the residual falls by 0.097 per cycle with
// Gauss-Seidel and 0.030 with 1.25 at 64^3.
constexpr float MG_OMEGA = PM_MG_OMEGA;

// ---------------------------------------------------------------------------
// Batched launches: one launch covers the blocks of several realisations.
// A table in device memory lists the member realisations' cumulative block
// counts; block b of the launch belongs to member q with off[q] <= b <
// off[q+1], and becomes block b - off[q] of that member's own grid (gx, gy,
// gz in its descriptor).  Blocks past off[m] and blocks of realisations
// whose `active` flag is 0 return at once, so a graph captured with the
// largest grid stays valid while the members' grids shrink.
// ---------------------------------------------------------------------------
constexpr int MAX_REAL = 64;
constexpr int MAX_MEMBERS = 2 * MAX_REAL;  // a realisation may appear twice in a table

struct BTable {
  int m;                       // members
  int off[MAX_MEMBERS + 1];    // cumulative block counts
};

// Planes per block of the batched mesh passes (colour pass, restriction,
// prolongation, warm-start prediction): a block's table lookup is shared by
// BZ planes of its (x, y) tile.
constexpr int BZ = 4;
template <class F>
__device__ __forceinline__ void each_plane(const BI& bi, int nz, F&& f) {
#pragma unroll 1
  for (int kk = 0; kk < BZ; ++kk) {
    BI b = bi;
    b.z = bi.z * BZ + kk;
    if (b.z >= nz) break;
    f(b);
  }
}

// The block of a batched launch -> member q of the table and its block
// coordinates (false: past the table's blocks, or an inactive realisation).
// The table's offsets are staged in shared memory by the whole block (one
// coalesced load) and searched there; every thread of the block must call.
template <class D>
__device__ __forceinline__ bool batch_map(const D* d, const BTable* t, const int* active, int& q,
                                          BI& bi) {
  __shared__ int s_off[MAX_MEMBERS + 1];
  const int tid = (int)(threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z));
  const int nth = (int)(blockDim.x * blockDim.y * blockDim.z);
  const int m = t->m;
  for (int i = tid; i <= m; i += nth) s_off[i] = t->off[i];
  __syncthreads();
  const int b = (int)blockIdx.x;
  if (m <= 0 || b >= s_off[m]) return false;
  int lo = 0, hi = m - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (s_off[mid] <= b) lo = mid; else hi = mid - 1;
  }
  q = lo;
  const D& e = d[lo];
  if (active && !active[e.r]) return false;
  const int lb = b - s_off[lo];
  bi = BI{lb % e.gx, (lb / e.gx) % e.gy, lb / (e.gx * e.gy), e.gx, e.gy, e.gz};
  return true;
}

}  // namespace pm
