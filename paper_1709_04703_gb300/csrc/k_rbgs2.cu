// The fused two-sweep red-black SOR smoother of the multigrid
// solve (Sec. 2.1, Eq. 3, cell units) for the large levels: one pass over
// the grid does red, black, red, black.  Tile heights 16, 24 and 32 give the
// same bits; the solve picks the fastest for each level-0 side.
#include "mg_arith.cuh"
#include "pm_kernels.cuh"

namespace pm {

// ---------------------------------------------------------------------------
// Two red-black SOR sweeps (red, black, red, black) in one pass: win -> wout.
//
// A CTA owns a 32 x TY tile of (x, y) (TY = 16, 24 or 32) and a chunk of zc
// planes and marches z.  Each of its 20 (TY + 8) threads (480, 640, 800) owns
// a pair of x-adjacent columns of the tile + 4-cell halo (40 x (TY + 8)
// cells) and keeps their values on planes t-4 .. t+1
// (and b on t-3 .. t) in registers; a ring of 5 planes in shared memory
// exposes them to the neighbouring columns.  Step t updates
//   red   on plane t   over the tile + 3   (old black values),
//   black on plane t-1 over the tile + 2,
//   red   on plane t-2 over the tile + 1,
//   black on plane t-3 over the tile       (final: stored),
// one cell of each pair per stage (the pair holds one cell of each colour).
// Within a step no stage reads a shared-memory value written in the same
// step (x/y neighbours live on the stage's own plane, written one step
// earlier; z neighbours are the thread's own registers), so one barrier per
// step suffices.  Every update applies sor_value(old, gs_value(..)) to the
// values the four one-colour launches would give it: the same bits.  win and wout must be
// different arrays unless zero_start (win is then not read: the iterate
// starts at zero, ghosts included).  Open boundaries: ghost cells are read,
// never updated; periodic: coordinates wrap.  Needs s even.
// ---------------------------------------------------------------------------
namespace {
constexpr int F2_TX = 32, F2_H = 4;
constexpr int F2_W = F2_TX + 2 * F2_H;  // region width 40
constexpr int F2_PW = F2_W / 2;         // pairs per row
constexpr int F2_R = 8;        // shared ring depth (planes t-3 .. t+1 used; power of 2)
constexpr int F2_D = 6;        // prefetch distance
constexpr int F2_PR = 8;       // prefetch ring depth (>= F2_D + 2; power of 2)
// tile height ty: region 40 x (ty + 8), one thread per pair, floats per
// plane, dynamic shared memory; up to 512 threads two CTAs fit on an SM
__host__ __device__ constexpr int f2_nt(int ty) { return F2_PW * (ty + 2 * F2_H); }
__host__ __device__ constexpr int f2_pl(int ty) { return F2_W * (ty + 2 * F2_H); }
constexpr size_t f2_smem(int ty) {
  return sizeof(float) * (size_t)f2_pl(ty) * (F2_R + 2 * F2_PR);
}
__host__ __device__ constexpr int f2_ctas_per_sm(int ty) { return f2_nt(ty) <= 512 ? 2 : 1; }

__device__ __forceinline__ void cp_async4(float* smem, const float* gmem, bool valid) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(sa), "l"(gmem),
               "r"(valid ? 4 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
}  // namespace

// Registers hold each plane of the pair in colour order: R the red cell
// ((x + y + p) even), K the black one; the red cell sits at x offset
// r(p) = (y + p) & 1 of the pair.  A cell's z neighbours have the other
// colour and the same x, i.e. the other register of the planes above and
// below.  The in-pair x neighbour is the partner register; the other x
// neighbour is in shared memory at offset -1 (cell at offset 0) or +2.  The
// four stages of step t all update the cell at offset r(t) (the colours
// alternate along z), and the register ring of six planes is renamed
// statically by unrolling the step loop six times.
template <bool PERIODIC, bool SIMPLE, bool ZERO, bool MASK, int TY>
struct Rbgs2 {
  static constexpr int RING = 6;
  static constexpr int F2_TY = TY, F2_PL = f2_pl(TY);
  const Grid win, wout, b;
  const float h2, gam, d0;
  const int s, x0, y0, z0, z1, ly, lx0, y, xa, me;
  float* sp;
  float* pu;
  float* pb;
  int uoff[2], boff[2];
  unsigned rmask[2];  // bit h: the cell is updated by the stage covering tile + h
  bool out0, out1;    // this thread stores cell xa / xa + 1 of the tile's planes
  int par0;           // (y + first step) & 1: the parities below follow from it and J
  int zst0, zst1;     // steady steps: all four stages active in z
  // the next plane to prefetch: its index P, its z (wrapped when periodic)
  // and its offsets in win and b; the output offset of the next step's plane
  int iss_P, iss_z;
  long long iss_u, iss_b, out_off;
  float R[RING], K[RING], BR[RING], BK[RING];  // plane t-4+m in slot (j + m) % 6

  // asynchronous copy of u and b of plane iss_P for this pair into its
  // prefetch slot, then advance to the next plane
  __device__ void issue() {
    const int P = iss_P;
    const int sl = P & (F2_PR - 1);
    const bool zok = PERIODIC || (P >= -1 && P <= s);
    const float* gu = win.base - 1 - win.sy + (zok ? iss_u : 0ll);
    const float* gb = b.base - 1 - b.sy + (zok ? iss_b : 0ll);
    float* du = pu + sl * F2_PL + me;
    float* db = pb + sl * F2_PL + me;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      if (ZERO) {
        du[k] = 0.0f;
      } else {
        const bool ok = zok && uoff[k] >= 0;
        cp_async4(du + k, gu + (ok ? uoff[k] : 0), ok);
      }
      const bool okb = zok && boff[k] >= 0;
      cp_async4(db + k, gb + (okb ? boff[k] : 0), okb);
    }
    cp_async_commit();
    ++iss_P;
    iss_u += win.sz;
    iss_b += b.sz;
    if (PERIODIC && ++iss_z == s) {
      iss_z = 0;
      iss_u = 0;
      iss_b = 0;
    }
  }

  // the prefetched plane P (cells in x order) into colour-ordered slot Q;
  // r1: (y + P) & 1
  template <int Q>
  __device__ void take(int P, int r1) {
    constexpr int q = Q;
    const int sl = P & (F2_PR - 1);
    const float* du = pu + sl * F2_PL + me;
    const float* db = pb + sl * F2_PL + me;
    const float a = du[0], c = du[1], e = db[0], f = db[1];
    R[q] = r1 ? c : a;
    K[q] = r1 ? a : c;
    BR[q] = r1 ? f : e;
    BK[q] = r1 ? e : f;
  }

  template <int Q>
  __device__ void put(int p, int r) {  // plane p (slot Q) into the shared ring; r: (y + p) & 1
    constexpr int q = Q;
    float* d = sp + (p & (F2_R - 1)) * F2_PL + me;
    d[r] = R[q];
    d[1 - r] = K[q];
  }

  template <int J>
  __device__ void step(int t) {
    issue();  // plane t + F2_D + 1
    __syncthreads();
    const int kc = par0 ^ (J & 1);  // x offset of the cell updated by all four stages
    const int xo = kc ? 1 : -1;
    // z activity of the four stages (bit 3 - st), all on in the steady steps
    unsigned zb = 0xFu;
    if (t < zst0 || t > zst1) {
      zb = 0u;
#pragma unroll
      for (int st = 0; st < 4; ++st) {
        const int p = t - st;
        const bool zact =
            (st == 0 || (st == 1 ? p >= z0 - 2 : st == 2 ? (p >= z0 - 1 && p <= z1)
                                                          : (p >= z0 && p < z1))) &&
            (PERIODIC || (p >= 0 && p < s));
        zb |= (zact ? 1u : 0u) << (3 - st);
      }
    }
    const unsigned act = (kc ? rmask[1] : rmask[0]) & zb;
#pragma unroll
    for (int st = 0; st < 4; ++st) {
      const int p = t - st;
      const int m = 4 - st;
      const int q = (J + m) % RING, qm = (J + m - 1) % RING, qp = (J + m + 1) % RING;
      // (the ball solve updates only the cells of its mask, carried by b)
      if (((act >> (3 - st)) & 1u) && (!MASK || g_in(b, xa + kc, y, p))) {
        float* c = sp + (p & (F2_R - 1)) * F2_PL + me + kc;
        const float xv = c[xo], ym = c[-F2_W], yp = c[F2_W];
        float nv;
        if ((st & 1) == 0) {  // red: partner and z neighbours are black
          const float s0 = nb6(xv, K[q], ym, yp, K[qm], K[qp]);
          nv = sor_value(R[q], SIMPLE ? gs_value(s0, BR[q], h2, true, 6.0f)
                                      : gs_value(s0, BR[q], h2, false,
                                                 mg_diag(xa + kc, y, p, s, PERIODIC, gam, d0)));
          R[q] = nv;
        } else {              // black: partner and z neighbours are red
          const float s0 = nb6(xv, R[q], ym, yp, R[qm], R[qp]);
          nv = sor_value(K[q], SIMPLE ? gs_value(s0, BK[q], h2, true, 6.0f)
                                      : gs_value(s0, BK[q], h2, false,
                                                 mg_diag(xa + kc, y, p, s, PERIODIC, gam, d0)));
          K[q] = nv;
        }
        *c = nv;
      }
    }
    if (t - 3 >= z0 && t - 3 < z1) {
      constexpr int q1 = (J + 1) % RING;  // plane t-3
      const int r = kc ^ 1;               // (y + t - 3) & 1
      float* g = wout.base + out_off;
      if (out0) g[0] = r ? K[q1] : R[q1];
      if (out1) g[1] = r ? R[q1] : K[q1];
    }
    out_off += wout.sz;
    put<(J + 5) % RING>(t + 1, kc ^ 1);
    cp_async_wait<F2_D - 1>();
    take<J % RING>(t + 2, kc);  // the slot of plane t-4 takes plane t+2
  }
};

template <bool PERIODIC, bool SIMPLE, bool ZERO, bool MASK, int TY>
__global__ void __launch_bounds__(f2_nt(TY), f2_ctas_per_sm(TY))
    k_rbgs2(Grid win, Grid wout, Grid b, float h2, float gam, float d0, int zc) {
  constexpr int F2_TY = TY, F2_PL = f2_pl(TY);
  pdl_wait();
  pdl_release();
  extern __shared__ float f2_smem[];
  const int s = wout.s;
  const int ly = threadIdx.x / F2_PW, lx0 = 2 * (threadIdx.x - ly * F2_PW);
  const int x0 = blockIdx.x * F2_TX, y0 = blockIdx.y * F2_TY, z0 = blockIdx.z * zc;
  if (MASK) {
    // the ball solve (level 0): a tile without a mask cell has nothing to
    // update, and the iterate is zero outside the mask in every buffer
    auto lo2 = [&](int a, int n) {  // smallest |offset| over cells a .. a + n - 1
      const int a0 = b.mbase + 2 * a, a1 = b.mbase + 2 * (a + n - 1);
      return a0 > 0 ? a0 : (a1 < 0 ? -a1 : 1);
    };
    const int dx = lo2(x0, F2_TX), dy = lo2(y0, F2_TY), dz = lo2(z0, zc);
    if (dx * dx + dy * dy + dz * dz > b.mr) return;
  }
  Rbgs2<PERIODIC, SIMPLE, ZERO, MASK, TY> g{win,   wout, b,  h2, gam, d0, s, x0, y0, z0,
                                            min(z0 + zc, s), ly, lx0, y0 - F2_H + ly,
                                            x0 - F2_H + lx0, ly * F2_W + lx0};
  g.sp = f2_smem;
  g.pu = g.sp + F2_R * F2_PL;
  g.pb = g.pu + F2_PR * F2_PL;
  auto mc = [&](int v) -> int {
    if (PERIODIC) {
      v %= s;
      return v < 0 ? v + s : v;
    }
    return (v < -1 || v > s) ? -(1 << 30) : v;
  };
  {
    const int yy = mc(g.y);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int xx = mc(g.xa + k);
      const bool ok = xx >= -1 && yy >= -1;
      g.uoff[k] = ok ? (xx + 1) + (yy + 1) * win.sy : -1;
      g.boff[k] = ok ? (xx + 1) + (yy + 1) * b.sy : -1;
    }
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    unsigned mk = 0;
    const int lx = lx0 + k, x = g.xa + k;
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const bool in = lx >= F2_H - h && lx < F2_H + F2_TX + h && ly >= F2_H - h &&
                      ly < F2_H + F2_TY + h &&
                      (PERIODIC || (x >= 0 && x < s && g.y >= 0 && g.y < s));
      mk |= (in ? 1u : 0u) << h;
    }
    g.rmask[k] = mk;
  }
  const bool out_tile = ly >= F2_H && ly < F2_H + F2_TY && lx0 >= F2_H && lx0 < F2_H + F2_TX;
  g.out0 = out_tile && g.xa < s && g.y < s;
  g.out1 = out_tile && g.xa + 1 < s && g.y < s;
#pragma unroll
  for (int m = 0; m < 6; ++m) g.R[m] = g.K[m] = g.BR[m] = g.BK[m] = 0.0f;
  const int tz = z0 - 3;  // first step; it needs planes tz-1 .. tz+1
  g.par0 = (g.y + tz) & 1;
  g.zst0 = z0 + 3;
  g.zst1 = PERIODIC ? g.z1 + 2 : min(g.z1 + 2, s - 1);
  g.out_off = (long long)(tz - 3) * wout.sz + (g.xa + g.y * wout.sy);
  {
    const int P0 = tz - 1;
    const int zw = PERIODIC ? mc(P0) : P0;
    g.iss_P = P0;
    g.iss_z = zw;
    g.iss_u = (long long)zw * win.sz;
    g.iss_b = (long long)zw * b.sz;
  }
  for (int P = tz - 1; P <= tz + F2_D; ++P) g.issue();
  cp_async_wait<F2_D - 1>();  // groups tz-1 .. tz+1 have landed
  g.template take<3>(tz - 1, g.par0 ^ 1);
  g.template take<4>(tz, g.par0);
  g.template take<5>(tz + 1, g.par0 ^ 1);
  g.template put<4>(tz, g.par0);
  const int tend = g.z1 + 2;
  for (int t = tz; t <= tend; t += 6) {
    g.template step<0>(t);
    if (t + 1 <= tend) g.template step<1>(t + 1); else break;
    if (t + 2 <= tend) g.template step<2>(t + 2); else break;
    if (t + 3 <= tend) g.template step<3>(t + 3); else break;
    if (t + 4 <= tend) g.template step<4>(t + 4); else break;
    if (t + 5 <= tend) g.template step<5>(t + 5); else break;
  }
  cp_async_wait<0>();
}

// kernel attributes that must be set outside any stream capture
template <int TY>
static cudaError_t set_rbgs2_smem() {
  cudaError_t e = cudaSuccess;
  auto set = [&](auto k) {
    cudaError_t r =
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)f2_smem(TY));
    if (r != cudaSuccess) e = r;
  };
  set(k_rbgs2<false, false, false, false, TY>);
  set(k_rbgs2<false, false, true, false, TY>);
  set(k_rbgs2<false, true, false, false, TY>);
  set(k_rbgs2<false, true, true, false, TY>);
  set(k_rbgs2<true, true, false, false, TY>);
  set(k_rbgs2<true, true, true, false, TY>);
  set(k_rbgs2<true, false, false, false, TY>);
  set(k_rbgs2<true, false, true, false, TY>);
  if (TY == 16) {  // the ball solve's level 0 (tile height 16 only)
    set(k_rbgs2<false, true, false, true, 16>);
    set(k_rbgs2<false, true, true, true, 16>);
  }
  return e;
}

cudaError_t mg_prepare() {
  cudaError_t e = set_rbgs2_smem<16>();
  if (e == cudaSuccess) e = set_rbgs2_smem<24>();
  if (e == cudaSuccess) e = set_rbgs2_smem<32>();
  if (e == cudaSuccess) e = cmg_prepare();
  return e;
}

bool rbgs2_tile_ok(int ty) { return ty == 16 || ty == 24 || ty == 32; }

int rbgs2_zchunk(int s, int ty) {
  // long chunks (each costs 6 extra steps), but about two waves of CTAs
  const long long tiles = (long long)((s + F2_TX - 1) / F2_TX) * ((s + ty - 1) / ty);
  const long long slots = 152LL * f2_ctas_per_sm(ty);
  int zc = 64;
  while (zc > 8 && tiles * ((s + zc - 1) / zc) < slots) zc /= 2;
  return zc;
}

template <int TY>
static void launch_rbgs2_t(cudaStream_t st, Grid win, Grid wout, Grid b, float h2, int periodic,
                           float gam, bool zero_start, int zc, float d0) {
  const dim3 grid((unsigned)((wout.s + F2_TX - 1) / F2_TX), (unsigned)((wout.s + TY - 1) / TY),
                  (unsigned)((wout.s + zc - 1) / zc));
  const dim3 blk(f2_nt(TY));
  const size_t sm = f2_smem(TY);
  const bool simple = (periodic || gam == 0.0f) && d0 == 6.0f;
#define PM_RBGS2(P, S, Z) \
  launch_pdl(k_rbgs2<P, S, Z, false, TY>, grid, blk, sm, st, win, wout, b, h2, gam, d0, zc)
  if (periodic && simple) {
    if (zero_start) PM_RBGS2(true, true, true); else PM_RBGS2(true, true, false);
  } else if (periodic) {
    if (zero_start) PM_RBGS2(true, false, true); else PM_RBGS2(true, false, false);
  } else if (simple) {
    if (zero_start) PM_RBGS2(false, true, true); else PM_RBGS2(false, true, false);
  } else {
    if (zero_start) PM_RBGS2(false, false, true); else PM_RBGS2(false, false, false);
  }
#undef PM_RBGS2
}

void launch_rbgs2(cudaStream_t st, Grid win, Grid wout, Grid b, float h2, int periodic,
                  float gam, bool zero_start, int zc, float d0, int ty) {
  if (b.mbase || !rbgs2_tile_ok(ty)) ty = 16;  // the ball solve: tile height 16
  if (zc <= 0) zc = rbgs2_zchunk(wout.s, ty);
  if (b.mbase) {  // the ball solve's level 0 (open, diagonal 6); the mask comes with b
    const dim3 grid((unsigned)((wout.s + F2_TX - 1) / F2_TX), (unsigned)((wout.s + 15) / 16),
                    (unsigned)((wout.s + zc - 1) / zc));
    if (zero_start)
      launch_pdl(k_rbgs2<false, true, true, true, 16>, grid, dim3(f2_nt(16)), f2_smem(16), st,
                 win, wout, b, h2, gam, d0, zc);
    else
      launch_pdl(k_rbgs2<false, true, false, true, 16>, grid, dim3(f2_nt(16)), f2_smem(16), st,
                 win, wout, b, h2, gam, d0, zc);
  } else if (ty == 32) {
    launch_rbgs2_t<32>(st, win, wout, b, h2, periodic, gam, zero_start, zc, d0);
  } else if (ty == 24) {
    launch_rbgs2_t<24>(st, win, wout, b, h2, periodic, gam, zero_start, zc, d0);
  } else {
    launch_rbgs2_t<16>(st, win, wout, b, h2, periodic, gam, zero_start, zc, d0);
  }
  note_launch();
}

}  // namespace pm
