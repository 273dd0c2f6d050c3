// C ABI of libpmshrink: context, step orchestration (Table 2 order), the
// host-side FP64 schedule (conformal time, lightcone distance), and the
// standalone solve / deposit / power-spectrum entry points.
#include <cufft.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "pm_kernels.cuh"

using namespace pm;

namespace {
std::atomic<long long> g_launches{0};
}  // namespace

void pm::note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
bool pm::pdl_enabled() {
  static const bool on = getenv("PM_NO_PDL") == nullptr;
  return on;
}

namespace {

constexpr double C_OVER_H0 = 2997.92458;  // Mpc/h
constexpr int SRC_GRID = 1216;            // 152 SMs x 8 blocks
constexpr int COARSE_SWEEPS = 6;
constexpr int FUSED_MIN = 192;  // smallest level side smoothed by the fused pass
constexpr int LEVEL_SWEEPS = 2;  // pre- and post-smoothing sweeps on levels below the finest
constexpr size_t BGW_OFF = 128;  // byte offset of the background weights in bgm

// ---------------------------------------------------------------------------
// FP64 cosmology on the host.  tau(a) = int_0^a da'/(a'^2 E), H0 = 1, with
// a' = u^2: tau = int_0^sqrt(a) 2 du / sqrt(om + ol u^6), a smooth integrand
// integrated by composite 8-point Gauss-Legendre on 64 panels.
// ---------------------------------------------------------------------------
struct Quad {
  double x[8], w[8];
  Quad() {
    const int m = 8;
    for (int i = 0; i < m; ++i) {
      double z = std::cos(M_PI * (i + 0.75) / (m + 0.5));
      double dp = 0.0;
      for (int it = 0; it < 100; ++it) {
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= m; ++k) {
          double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
          p0 = p1;
          p1 = p2;
        }
        dp = m * (z * p1 - p0) / (z * z - 1.0);
        double dz = p1 / dp;
        z -= dz;
        if (std::fabs(dz) < 1e-16) break;
      }
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= m; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = m * (z * p1 - p0) / (z * z - 1.0);
      x[i] = z;
      w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
  }
};

double tau_of_a(double a, double om, double ol) {
  static const Quad q;
  const int panels = 64;
  double U = std::sqrt(a), hsz = U / panels, tot = 0.0;
  for (int p = 0; p < panels; ++p) {
    double c = (p + 0.5) * hsz, hw = 0.5 * hsz;
    for (int i = 0; i < 8; ++i) {
      double u = c + hw * q.x[i];
      tot += hw * q.w[i] * 2.0 / std::sqrt(om + ol * u * u * u * u * u * u);
    }
  }
  return tot;
}

double a_of_tau(double t, double om, double ol) {
  double lo = 1e-12, hi = 4.0;
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    if (tau_of_a(mid, om, ol) < t) lo = mid; else hi = mid;
    if (hi - lo <= 4e-16 * hi) break;
  }
  return 0.5 * (lo + hi);
}

bool mg_size_ok(int n) {
  if (n < 4) return false;
  while (n % 2 == 0) n /= 2;
  return n == 1 || n == 3;
}

// Smallest q * 2^j >= m with q in {1, 3, 5, 7}: sides that halve down to at
// most 7 for the multigrid (open cubes; the periodic box is the mesh itself).
int mg_round_up(int m) {
  int best = 1 << 30;
  for (int q : {1, 3, 5, 7}) {
    for (int p = q; p < (1 << 29); p *= 2) {
      if (p >= m) { best = std::min(best, p); break; }
    }
  }
  return best;
}

std::string g_err;  // last error of a context-free call

// NVTX range over a host scope (a step, a solve, a sort, a shrink), for
// timeline tools; inert when no tool is attached
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace

// a pair of profiling events around a launch group of one kernel class
struct Pend { int cls, e0, e1; double bytes; };

struct pm_ctx {
  pm_config cfg;
  cudaStream_t st = nullptr;
  int n = 0, P = 0;
  long long N0 = 0;
  std::vector<double> a, dtau, a_half, chi, R;
  int step = 0;

  float4 *pos = nullptr, *mom = nullptr, *pos2 = nullptr, *mom2 = nullptr;
  float4 *lc_pos = nullptr, *lc_mom = nullptr, *forces = nullptr;
  float4* grad = nullptr;  // gradient field of the potential, (n+2)^3
  long long n_active = 0, n_lc = 0;
  bool forces_valid = false;
  long long forces_n = 0;
  unsigned char* flags = nullptr;
  unsigned int* block_keep = nullptr;
  unsigned long long* keep_off = nullptr;

  unsigned long long* rho = nullptr;
  // potential as a double-float pair, two buffers: the defect evaluation
  // that applies a V-cycle's correction writes Phi + e out of place
  float* phi_h[2] = {nullptr, nullptr};
  float* phi_l[2] = {nullptr, nullptr};
  int cur = 0;
  float *f_hi = nullptr, *f_lo = nullptr;
  float *prev_hi = nullptr, *prev_lo = nullptr;  // previous step's solution
  int n_sol = 0;            // consecutive warm-startable solutions
  double ah_hist[2] = {0, 0};  // a_half of the last two solves
  std::vector<float*> lu, lb;   // level arrays (compact padded); level 0 for e / r
  std::vector<float*> lu2;      // second iterate per level (u + P uc before post-smoothing)
  std::vector<int> ls;          // level sides of the current cube

  double* partial = nullptr;    // per-block FP64 partial sums
  void* partial_m = nullptr;    // per-block int128 moments
  unsigned int* counter = nullptr;
  double* d_scal = nullptr;     // [0] ||f||^2, [1..10] moments, [11] ||r||^2, [12] sum phi
  double* bgm = nullptr;        // background moments (10), then at BGW_OFF the weights
  df* bgw = nullptr;            // per-axis mean-density weights w_g, g in [0, n)
  float* ballw = nullptr;       // spherical keep region: mean-density image, n^3
  SortWork sortw{};             // particle order by cell (sort_every > 0)
  long long n_allocs = 0;       // device allocations so far (fault injection)
  // PM_FP64_PLAIN: the potential and source in double (full (n+2)^3) and
  // the coarse levels (compact, level 0 unused)
  double *phi64 = nullptr, *f64 = nullptr;
  std::vector<double*> lu64, lb64;
  // PM_MIXED_FP64: phi64 is the potential of the run (full (n+2)^3, its
  // ghost layer the open boundary's values) and prev64 the previous step's
  // solution for the warm start; f64 the source of the current solve
  double* prev64 = nullptr;
  BallRule ball_rule{};         // its Gauss-Legendre rule
  std::vector<unsigned char> h_bg;  // host image of bgm + bgw
  unsigned long long* d_cnt = nullptr;  // [0] n_keep, [1] escaped
  int* d_overflow = nullptr;
  double* h_scal = nullptr;     // pinned mirrors
  unsigned long long* h_cnt = nullptr;

  int lo = 0, s = 0, periodic = 1;
  bool cube_valid = false;
  // PM_DOMAIN_BALL in the open phase: the mask of the current cube (Grid's
  // mask fields; mbase = 0: no mask)
  int mbase = 0, mr = 0;
  double ball_rm = 0.0;  // its radius R + 2 (cells)

  // CUDA graph of one V-cycle for the current cube and level-0 grids (needs a
  // non-default stream to capture on)
  bool use_graphs = false;
  bool capturing = false;
  int ev_graph_next = 0;
  // (one graph per level-0 start: from zero, and from the iterate)
  struct VGraph {
    bool valid = false;
    int lo = 0, s = 0, per = 0, prof = 0, zero0 = 0, mr = 0;
    float *u0 = nullptr, *b0 = nullptr;
    cudaGraphExec_t exec = nullptr;
    long long kernels = 0;
    std::vector<struct Pend> pend;  // event pairs recorded inside the graph
  } vg[2];
  // the fused smoother's tile height and z chunk per level side (tune_fused)
  struct F2Pick {
    int s, ty, zc;
  };
  std::vector<F2Pick> f2_pick;
  // the mixed forms' level-0 correction e of A e = r (compact (n+2)^3; its
  // ghost layer stays zero: homogeneous Dirichlet for the correction)
  float* ecorr = nullptr;

  // per-class event timing (pm_profile)
  bool prof_on = false;
  std::vector<cudaEvent_t> ev;
  int ev_next = 0;
  std::vector<Pend> pend;
  std::vector<Pend> pend_graph;  // event pairs recorded inside the V-cycle graph
  double prof_ms[PM_PROF_N] = {0};
  long long prof_groups[PM_PROF_N] = {0};
  double prof_bytes[PM_PROF_N] = {0};
  long long prof_lost = 0;

  // learned initial guess (not owned) and its dense scratch fields
  pm_guess* net = nullptr;
  float *nn_in = nullptr, *nn_out = nullptr;
  int guess_used_last = 0;
  long long guess_used_total = 0;
  // training-pair capture targets (caller's device memory)
  float *cap_r = nullptr, *cap_e = nullptr;

  // diffusion gravity: diagonal shift of the current solve (0: Poisson) and
  // whether the field holds the state of the last step
  float sig = 0.0f;       // in the FP32 V-cycle (preconditioner)
  double sig_d = 0.0;     // in the double-float defect and right-hand side
  bool field_ready = false;

  int vcycles_last = 0;
  int vc_prev = 0;          // V-cycles of the previous solve
  long long vcycles_total = 0;
  double resid_last = 0.0;
  double resid_start = 0.0, resid_guess = 0.0;  // of the last solve
  long long particle_steps = 0;
  std::string err;
};

namespace {

pm_status fail(pm_ctx* c, pm_status code, const std::string& msg) {
  if (c) c->err = msg; else g_err = msg;
  return code;
}

#define CK(call)                                                                   \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess)                                                         \
      return fail(ctx, PM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define CKL()                                                                      \
  do {                                                                             \
    cudaError_t e_ = cudaGetLastError();                                           \
    if (e_ != cudaSuccess)                                                         \
      return fail(ctx, PM_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e_)); \
  } while (0)

Grid full_view(const pm_ctx* c, float* base, int lo, int s) {
  Grid g{};
  g.sy = c->P;
  g.sz = c->P * c->P;
  g.s = s;
  g.base = base + (lo + 1) + (lo + 1) * g.sy + (lo + 1) * g.sz;
  return g;
}

Grid compact_view(float* base, int s) {
  Grid g{};
  g.sy = s + 2;
  g.sz = (s + 2) * (s + 2);
  g.s = s;
  g.base = base + 1 + g.sy + g.sz;
  return g;
}

// g with the ball solve's mask of level l of the current cube (if any)
Grid masked(const pm_ctx* c, Grid g, int l) {
  if (c->mbase) {
    g.mbase = c->mbase;
    g.mstep = 2 << l;
    g.mr = c->mr;
    g.mrm2 = (float)(c->ball_rm * c->ball_rm);
    g.mrb2 = (float)((c->ball_rm + 0.5) * (c->ball_rm + 0.5));
  }
  return g;
}

bool is_open(const pm_ctx* c, double R) {
  if (c->cfg.bc == PM_BC_OPEN) return true;
  if (c->cfg.bc == PM_BC_PERIODIC) return false;
  return R <= 0.5 * c->n - 1.0;
}

// Keep test of radius R (the cube's float bounds are passed separately).
KeepBall keep_ball(const pm_ctx* c, double R) {
  return KeepBall{c->cfg.domain != PM_DOMAIN_CUBE ? 1 : 0, 0.5 * c->n, R * R};
}

// m-point Gauss-Legendre rule on [0, 1] (Newton on the Legendre recurrence)
// with each weight times the tent 1 - xi.
BallRule ball_rule() {
  BallRule r{};
  const int m = BALL_GL;
  for (int i = 0; i < m; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (m + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= m; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = m * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= m; ++k) {
      const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    dp = m * (z * p1 - p0) / (z * z - 1.0);
    const double w = 2.0 / ((1.0 - z * z) * dp * dp);
    const double xi = 0.5 * (z + 1.0);
    r.xi[i] = (float)xi;
    r.om[i] = (float)(0.5 * w * (1.0 - xi));
  }
  return r;
}

// Active mesh cube for keep half-width R (see pm_config.bc).
void geometry(const pm_ctx* c, double R, int* lo, int* s, int* periodic) {
  const int n = c->n;
  if (!is_open(c, R)) { *lo = 0; *s = n; *periodic = 1; return; }
  *periodic = 0;
  if (R > 0.5 * n - 1.0) { *lo = 0; *s = n; return; }
  // the assignment reaches one cell (CIC) or two (TSC) beyond the keep cube;
  // the ball solve's mask two beyond the keep radius and its ghosts one more
  const int reach = c->cfg.domain == PM_DOMAIN_BALL ? 3
                    : c->cfg.assignment == PM_ASSIGN_TSC ? 2 : 1;
  int m = (int)std::ceil(R) + reach;
  int side = std::min(mg_round_up(2 * m), n);
  *s = side;
  *lo = n / 2 - side / 2;
}

// The fused smoother's launch shape for a level of side s: the tuned pick,
// else tile height 16 with the default z chunk.
void f2_choice(const pm_ctx* c, int s, int* ty, int* zc) {
  *ty = 16;
  *zc = 0;
  for (const auto& p : c->f2_pick)
    if (p.s == s) {
      *ty = p.ty;
      *zc = p.zc;
    }
}

// Time the fused smoother's launch shapes (tile height 16, 24, 32; z chunk
// by rule, 64, 128) on every level side >= FUSED_MIN that the run's cubes
// give, and keep the fastest per side.  All shapes give the same bits, so
// the pick changes the speed only.  The run's cubes follow from the
// schedule alone (geometry), so this runs once, at init, on the level-0
// scratch grids (cleared here; set_cube clears them again).  The ball
// solve keeps tile height 16; FP64 everywhere has no fused pass.
cudaError_t tune_fused(pm_ctx* ctx) {
  ctx->f2_pick.clear();
  if (ctx->cfg.domain == PM_DOMAIN_BALL || ctx->cfg.precision == PM_FP64_PLAIN ||
      ctx->lu.empty())
    return cudaSuccess;
  std::vector<int> sides;
  for (size_t k = 0; k < ctx->R.size(); ++k) {
    int lo, s, per;
    geometry(ctx, ctx->R[k], &lo, &s, &per);
    for (int l = s; l >= FUSED_MIN && l % 2 == 0; l /= 2)
      if (std::find(sides.begin(), sides.end(), l) == sides.end()) sides.push_back(l);
  }
  if (sides.empty()) return cudaSuccess;
  const size_t bytes = sizeof(float) * (size_t)(ctx->n + 2) * (ctx->n + 2) * (ctx->n + 2);
  cudaError_t e = cudaSuccess;
  for (float* p : {ctx->lu[0], ctx->lu2[0], ctx->lb[0]})
    if (e == cudaSuccess) e = cudaMemsetAsync(p, 0, bytes, ctx->st);
  if (e != cudaSuccess) return e;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess) return e;
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
    cudaEventDestroy(e0);
    return e;
  }
  for (int s : sides) {
    const Grid u = compact_view(ctx->lu[0], s), w = compact_view(ctx->lu2[0], s);
    const Grid b = compact_view(ctx->lb[0], s);
    float best = 1e30f;
    pm_ctx::F2Pick pick{s, 16, 0};
    for (int ty : {16, 24, 32})
      for (int zq : {0, 64, 128}) {
        const int zc = zq > 0 ? zq : rbgs2_zchunk(s, ty);
        if (zq > 0 && (zc >= s || zc == rbgs2_zchunk(s, ty))) continue;
        // one pass from the iterate (u -> w), as the post-smoothing runs:
        // one to warm up, three timed
        launch_rbgs2(ctx->st, u, w, b, 1.0f, 0, 0.0f, false, zc, 6.0f, ty);
        cudaEventRecord(e0, ctx->st);
        for (int r = 0; r < 3; ++r)
          launch_rbgs2(ctx->st, u, w, b, 1.0f, 0, 0.0f, false, zc, 6.0f, ty);
        cudaEventRecord(e1, ctx->st);
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
          best = ms;
          pick = {s, ty, zc};
        }
      }
    if (e != cudaSuccess) break;
    ctx->f2_pick.push_back(pick);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  return e;
}

// Exact float bounds [klo, khi] with x in it  <=>  |(double)x - c| <= R.
void keep_bounds(double c, double R, float* klo, float* khi) {
  float l = (float)(c - R);
  while ((double)l - c < -R) l = std::nextafter(l, INFINITY);
  while ((double)std::nextafter(l, -INFINITY) - c >= -R) l = std::nextafter(l, -INFINITY);
  float h = (float)(c + R);
  while ((double)h - c > R) h = std::nextafter(h, -INFINITY);
  while ((double)std::nextafter(h, INFINITY) - c <= R) h = std::nextafter(h, INFINITY);
  *klo = l;
  *khi = h;
}

// Integral of the CIC tent max(0, 1 - |t|) over t < u.
static double tent_integral(double u) {
  if (u <= -1.0) return 0.0;
  if (u <= 0.0) return 0.5 * (u + 1.0) * (u + 1.0);
  if (u <= 1.0) return 1.0 - 0.5 * (1.0 - u) * (1.0 - u);
  return 1.0;
}

// Integral of the TSC kernel (3/4 - t^2 on |t| <= 1/2, (3/2 - |t|)^2 / 2 on
// 1/2 <= |t| <= 3/2) over t < u.
static double tsc_integral(double u) {
  if (u <= -1.5) return 0.0;
  if (u <= -0.5) return (1.5 + u) * (1.5 + u) * (1.5 + u) / 6.0;
  if (u <= 0.5) return 1.0 / 6.0 + 0.75 * (u + 0.5) - (u * u * u + 0.125) / 3.0;
  if (u <= 1.5) return 1.0 - (1.5 - u) * (1.5 - u) * (1.5 - u) / 6.0;
  return 1.0;
}

pm_status set_cube(pm_ctx* ctx, int lo, int s, int periodic, double R) {
  bool same = ctx->cube_valid && lo == ctx->lo && s == ctx->s && periodic == ctx->periodic;
  ctx->lo = lo;
  ctx->s = s;
  ctx->periodic = periodic;
  ctx->cube_valid = true;
  // the ball solve's mask: cell centres within R + 2 of c; twice a centre's
  // offset from c along an axis is the odd integer 2 (lo + i) + 1 - n, and
  // the mask holds the squares' sum up to floor(4 (R + 2)^2)
  const int mbase0 = ctx->mbase, mr0 = ctx->mr;
  ctx->mbase = 0;
  ctx->mr = 0;
  if (ctx->cfg.domain == PM_DOMAIN_BALL && !periodic && R < (double)ctx->n) {
    const double rm = R + 2.0;
    ctx->mbase = 2 * lo + 1 - ctx->n;
    ctx->mr = (int)std::floor(rm * rm * 4.0);
    ctx->ball_rm = rm;
  }
  // the correction is zero outside the mask (the masked passes never write
  // there, and the defect adds it everywhere): cleared when the mask moves
  if (same && ctx->ecorr && (ctx->mbase != mbase0 || ctx->mr != mr0))
    CK(cudaMemsetAsync(ctx->ecorr, 0, sizeof(float) * (size_t)(s + 2) * (s + 2) * (s + 2),
                       ctx->st));
  // mean-density term of delta: per axis the image of the keep interval
  // [c - R, c + R] under the assignment kernel (CIC tent or TSC),
  // w_g = T(c + R - x_g) - T(c - R - x_g) at x_g = g + 1/2 with T the
  // kernel's integral (ones when periodic), and its moments about c
  // (separable sums)
  const int n = ctx->n;
  double* h = (double*)ctx->h_bg.data();
  df* hw = (df*)(ctx->h_bg.data() + BGW_OFF);
  const double c = 0.5 * n;
  double W0 = 0.0, W1 = 0.0, W2 = 0.0;
  for (int g = 0; g < n; ++g) {
    const double x = g + 0.5;
    const bool tsc = ctx->cfg.assignment == PM_ASSIGN_TSC;
    const double w = periodic ? 1.0
                     : tsc    ? tsc_integral((c + R) - x) - tsc_integral((c - R) - x)
                              : tent_integral((c + R) - x) - tent_integral((c - R) - x);
    hw[g].hi = (float)w;
    hw[g].lo = (float)(w - (double)hw[g].hi);
    if (g >= lo && g < lo + s) {
      const double y = x - c;
      W0 += w;
      W1 += w * y;
      W2 += w * y * y;
    }
  }
  const double W00 = W0 * W0;
  const double mom[10] = {W00 * W0, W00 * W1, W00 * W1, W00 * W1, W00 * W2, W00 * W2, W00 * W2,
                          W0 * W1 * W1, W0 * W1 * W1, W0 * W1 * W1};
  std::memcpy(h, mom, sizeof(mom));
  CK(cudaMemcpyAsync(ctx->bgm, ctx->h_bg.data(), ctx->h_bg.size(), cudaMemcpyHostToDevice,
                     ctx->st));
  if (ctx->ballw && !periodic)  // spherical keep region: image of the ball and its moments
    launch_ball_w(ctx->st, ctx->ballw, n, lo, s, R, ctx->ball_rule, ctx->partial, ctx->counter,
                  ctx->bgm);
  if (same) return PM_OK;
  // multigrid level sides: halve while > 4
  ctx->ls.clear();
  int sl = s;
  ctx->ls.push_back(sl);
  while (sl > 4 && sl % 2 == 0) {
    sl /= 2;
    ctx->ls.push_back(sl);
  }
  if (sl > 8) return fail(ctx, PM_EINVAL, "cube side does not coarsen to <= 8");
  if (ctx->ecorr)  // the correction's ghost layer (zero) moves with the side
    CK(cudaMemsetAsync(ctx->ecorr, 0,
                       sizeof(float) * (size_t)(s + 2) * (s + 2) * (s + 2), ctx->st));
  for (size_t l = 0; l < ctx->ls.size(); ++l) {
    size_t bytes = sizeof(float) * (size_t)(ctx->ls[l] + 2) * (ctx->ls[l] + 2) * (ctx->ls[l] + 2);
    CK(cudaMemsetAsync(ctx->lu[l], 0, bytes, ctx->st));
    CK(cudaMemsetAsync(ctx->lb[l], 0, bytes, ctx->st));
    CK(cudaMemsetAsync(ctx->lu2[l], 0, bytes, ctx->st));
    if (l > 0 && l < ctx->lu64.size() && ctx->lu64[l]) {
      CK(cudaMemsetAsync(ctx->lu64[l], 0, 2 * bytes, ctx->st));
      CK(cudaMemsetAsync(ctx->lb64[l], 0, 2 * bytes, ctx->st));
    }
  }
  return PM_OK;
}

// Event pairs around launch groups; elapsed times are collected after the
// next stream synchronisation.
void prof_flush(pm_ctx* ctx) {
  for (const auto& p : ctx->pend) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ctx->ev[p.e0], ctx->ev[p.e1]) == cudaSuccess) {
      ctx->prof_ms[p.cls] += ms;
      ctx->prof_groups[p.cls] += 1;
      ctx->prof_bytes[p.cls] += p.bytes;
    } else {
      cudaGetLastError();  // a timing failure must not surface as a launch error
      ctx->prof_lost += 1;
    }
  }
  ctx->pend.clear();
  ctx->ev_next = 0;
}

constexpr int EV_POOL = 1024;  // events [0, EV_POOL) eager, [EV_POOL, 2 EV_POOL) graph

int prof_begin(pm_ctx* ctx) {
  if (!ctx->prof_on) return -1;
  if (ctx->capturing) {
    if ((ctx->ev_graph_next - EV_POOL) % (EV_POOL / 2) + 2 > EV_POOL / 2) return -1;
    int e = ctx->ev_graph_next++;
    // inside a capture only an external record becomes a real event node
    cudaEventRecordWithFlags(ctx->ev[e], ctx->st, cudaEventRecordExternal);
    return e;
  }
  if (ctx->ev_next + 2 > EV_POOL) {
    cudaStreamSynchronize(ctx->st);
    prof_flush(ctx);
  }
  int e = ctx->ev_next++;
  cudaEventRecord(ctx->ev[e], ctx->st);
  return e;
}

void prof_end(pm_ctx* ctx, int cls, int e0, double bytes) {
  if (e0 < 0) return;
  if (ctx->capturing) {
    int e1 = ctx->ev_graph_next++;
    cudaEventRecordWithFlags(ctx->ev[e1], ctx->st, cudaEventRecordExternal);
    ctx->pend_graph.push_back({cls, e0, e1, bytes});
    return;
  }
  int e1 = ctx->ev_next++;
  cudaEventRecord(ctx->ev[e1], ctx->st);
  ctx->pend.push_back({cls, e0, e1, bytes});
}

pm_status sync_read(pm_ctx* ctx) {
  CK(cudaMemcpyAsync(ctx->h_scal, ctx->d_scal, sizeof(double) * 16, cudaMemcpyDeviceToHost,
                     ctx->st));
  CK(cudaMemcpyAsync(ctx->h_cnt, ctx->d_cnt, sizeof(unsigned long long) * 4,
                     cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  if (ctx->prof_on) prof_flush(ctx);
  return PM_OK;
}

// V(2,2) cycle on level 0 grids (u0, b0) of the current cube.
// Two red-black SOR sweeps (red, black, red, black) on a level; zero_start
// when the iterate is known to be zero on entry (not necessarily stored).
void smooth2(pm_ctx* ctx, Grid u, Grid b, float h2, int per, float g, bool zero_start,
             float d0, int sweeps = 2) {
  for (int sw = 0; sw < sweeps; ++sw) {
    launch_rbgs(ctx->st, u, b, h2, 0, per, g, zero_start && sw == 0 ? 1 : 0, d0);
    launch_rbgs(ctx->st, u, b, h2, 1, per, g, zero_start && sw == 0 ? 2 : 0, d0);
  }
}

// V(2,2) cycle on level-0 grids (u0, b0).  On levels of side >= FUSED_MIN
// the two pre- and two post-smoothing sweeps are each one fused pass
// (k_rbgs2): the pre-smoothing starts from zero on every level but, in the
// plain path, the finest one, where it writes a scratch grid instead of u0;
// the prolongation writes u + P uc to a second grid that the post-smoothing
// reads back into u.  Smaller levels take four one-colour passes in place.
pm_status vcycle(pm_ctx* ctx, Grid u0, Grid b0, bool zero0) {
  const int per = ctx->periodic;
  const int L = (int)ctx->ls.size() - 1;
  Grid U[16], B[16], Upre[16];
  if (L >= 16) return fail(ctx, PM_EINVAL, "too many multigrid levels");
  // the ball solve: every level masked, homogeneous coarse ghosts (gam 0)
  const bool ball = ctx->mbase != 0;
  U[0] = masked(ctx, u0, 0);
  B[0] = masked(ctx, b0, 0);  // (the fused smoother reads the mask from b)
  for (int l = 1; l <= L; ++l) {
    U[l] = masked(ctx, compact_view(ctx->lu[l], ctx->ls[l]), l);
    B[l] = masked(ctx, compact_view(ctx->lb[l], ctx->ls[l]), l);
  }
  const double c0 = (double)ctx->s * ctx->s * ctx->s;
  // algorithmic bytes per fine cell: a red-black SOR sweep reads u
  // and b and writes u, 12 B per sweep (two sweeps per smoothing: 24; the
  // fused pass moves 8 from a zero start and 12 otherwise, since its two
  // sweeps share one read and one write); residual + restriction reads u
  // and b and writes the coarse b and u (9); prolongation reads u and the
  // coarse u and writes u + P uc (8.5)
  float h2 = 1.0f;
  int ec = -1;
  // open-boundary ghost factor of level l (spacing H = 2^l), see k_mg.cu
  auto gam = [&](int l) {
    float H = (float)(1 << l);
    return ball ? 0.0f : (H - 1.0f) / (H + 1.0f);
  };
  // the levels from the first of side <= cmg_top_side run in one
  // thread-block cluster (k_cmg.cu)
  int Lc = 0;
  while (Lc < L && ctx->ls[Lc] > cmg_top_side(ball ? 1 : cmg_cluster())) ++Lc;
  for (int l = 0; l < Lc; ++l) {
    int e = l == 0 ? prof_begin(ctx) : -1;
    // below level 0 the restriction zeroes the coarse iterate
    const bool zs = l == 0 ? zero0 : true;
    const bool fused = ctx->ls[l] >= FUSED_MIN && (!ball || l == 0);
    const float d0 = 6.0f + ctx->sig * h2;  // h2 = 4^l
    Upre[l] = (zs || !fused) ? U[l] : compact_view(ctx->lu[0], ctx->ls[0]);
    if (fused && !zs && !per)  // the scratch grids take u0's Dirichlet ghost values
      launch_copy_ghosts(ctx->st, U[0], Upre[0], compact_view(ctx->lu2[0], ctx->ls[0]));
    int f2_ty = 16, f2_zc = 0;
    f2_choice(ctx, ctx->ls[l], &f2_ty, &f2_zc);
    if (fused)
      launch_rbgs2(ctx->st, U[l], Upre[l], B[l], h2, per, gam(l), zs, f2_zc, d0, f2_ty);
    else
      smooth2(ctx, U[l], B[l], h2, per, gam(l), zs, d0, l > 0 ? LEVEL_SWEEPS : 2);
    if (l == 0) {
      prof_end(ctx, PM_PROF_SMOOTH0, e, 24.0 * c0);
      e = prof_begin(ctx);
    }
    launch_resid_restrict(ctx->st, Upre[l], B[l], 1.0f / h2, U[l + 1], B[l + 1], per, gam(l),
                          d0);
    if (l == 0) {
      prof_end(ctx, PM_PROF_TRANSFER0, e, 9.0 * c0);
      ec = prof_begin(ctx);
    }
    h2 *= 4.0f;
  }
  if (Lc == 0) ec = prof_begin(ctx);
  launch_cmg(ctx->st, U[Lc], B[Lc], Lc, per, COARSE_SWEEPS, Lc == 0 ? zero0 : true,
                   ctx->sig);
  for (int l = Lc - 1; l >= 0; --l) {
    h2 *= 0.25f;
    int e = -1;
    if (l == 0) {
      prof_end(ctx, PM_PROF_COARSE, ec, (Lc > 0 ? 8.0 / 7.0 * 81.0 * c0 / 8.0 : 0.0));
      e = prof_begin(ctx);
    }
    const bool fused = ctx->ls[l] >= FUSED_MIN && (!ball || l == 0);
    const float d0 = 6.0f + ctx->sig * h2;
    Grid W = compact_view(ctx->lu2[l], ctx->ls[l]);
    if (fused)
      launch_prolong_to(ctx->st, U[l + 1], Upre[l], W, per, gam(l + 1));
    else
      launch_prolong(ctx->st, U[l + 1], U[l], per, gam(l + 1));
    if (l == 0) {
      prof_end(ctx, PM_PROF_TRANSFER0, e, 8.5 * c0);
      e = prof_begin(ctx);
    }
    int f2_ty = 16, f2_zc = 0;
    f2_choice(ctx, ctx->ls[l], &f2_ty, &f2_zc);
    if (fused)
      launch_rbgs2(ctx->st, W, U[l], B[l], h2, per, gam(l), false, f2_zc, d0, f2_ty);
    else
      smooth2(ctx, U[l], B[l], h2, per, gam(l), false, d0, l > 0 ? LEVEL_SWEEPS : 2);
    if (l == 0) prof_end(ctx, PM_PROF_SMOOTH0, e, 24.0 * c0);
  }
  if (Lc == 0) prof_end(ctx, PM_PROF_COARSE, ec, 0.0);
  CKL();
  return PM_OK;
}

void drop_graph(pm_ctx* ctx) {
  for (auto& g : ctx->vg) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g = pm_ctx::VGraph();
  }
}

// One V-cycle: replay of a graph captured for the current cube / grids, or
// eager launches when the context's stream cannot be captured.
pm_status vcycle_run(pm_ctx* ctx, Grid u0, Grid b0, bool zero0) {
  // the diffusion substeps change the shift every solve: no graph for them
  if (!ctx->use_graphs || ctx->sig != 0.0f) return vcycle(ctx, u0, b0, zero0);
  auto& g = ctx->vg[zero0 ? 1 : 0];
  if (!(g.valid && g.lo == ctx->lo && g.s == ctx->s && g.per == ctx->periodic &&
        g.u0 == u0.base && g.b0 == b0.base && g.prof == (int)ctx->prof_on &&
        g.zero0 == (int)zero0 && g.mr == ctx->mr)) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g = pm_ctx::VGraph();
    CK(cudaStreamBeginCapture(ctx->st, cudaStreamCaptureModeThreadLocal));
    ctx->capturing = true;
    ctx->ev_graph_next = EV_POOL + (zero0 ? EV_POOL / 2 : 0);
    ctx->pend_graph.clear();
    long long l0 = g_launches.load();
    pm_status st = vcycle(ctx, u0, b0, zero0);
    ctx->capturing = false;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(ctx->st, &graph);
    long long nk = g_launches.load() - l0;
    g_launches.fetch_sub(nk);
    if (st != PM_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (e != cudaSuccess)
      return fail(ctx, PM_ECUDA, std::string("V-cycle capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess)
      return fail(ctx, PM_ECUDA, std::string("V-cycle instantiate: ") + cudaGetErrorString(e));
    g.valid = true;
    g.lo = ctx->lo;
    g.s = ctx->s;
    g.per = ctx->periodic;
    g.u0 = u0.base;
    g.b0 = b0.base;
    g.prof = ctx->prof_on;
    g.zero0 = zero0;
    g.mr = ctx->mr;  // the ball's mask radius (captured in the kernels' grids)
    g.kernels = nk;
    g.pend = ctx->pend_graph;
  }
  CK(cudaGraphLaunch(g.exec, ctx->st));
  g_launches.fetch_add(g.kernels);
  if (ctx->prof_on) ctx->pend.insert(ctx->pend.end(), g.pend.begin(), g.pend.end());
  return PM_OK;
}

// Iterate to rtol.  f2 = ||f||^2 already in d_scal[0] (read at first sync).
// With a learned guess, the first correction comes from the network applied
// to the residual of the start instead of from a V-cycle.
GridD full_view64(const pm_ctx* c, double* base, int lo, int s) {
  GridD g;
  g.sy = c->P;
  g.sz = c->P * c->P;
  g.s = s;
  g.base = base + (lo + 1) + (lo + 1) * g.sy + (lo + 1) * g.sz;
  return g;
}

GridD compact_view64(double* base, int s) {
  GridD g;
  g.sy = s + 2;
  g.sz = (s + 2) * (s + 2);
  g.s = s;
  g.base = base + 1 + g.sy + g.sz;
  return g;
}

// V(2,2) in double on the level-0 grids (u0, b0): the FP32 cycle's order and
// boundary treatment, one-colour passes on every level, 64 sweeps at the
// coarsest level (side <= 8)
pm_status vcycle64(pm_ctx* ctx, GridD u0, GridD b0) {
  const int per = ctx->periodic;
  const int L = (int)ctx->ls.size() - 1;
  if (L >= 16) return fail(ctx, PM_EINVAL, "too many multigrid levels");
  GridD U[16], B[16];
  U[0] = u0;
  B[0] = b0;
  for (int l = 1; l <= L; ++l) {
    U[l] = compact_view64(ctx->lu64[l], ctx->ls[l]);
    B[l] = compact_view64(ctx->lb64[l], ctx->ls[l]);
  }
  auto gam = [&](int l) {
    const double H = (double)(1 << l);
    return per ? 0.0 : (H - 1.0) / (H + 1.0);
  };
  auto smooth = [&](int l, double h2) {
    for (int sw = 0; sw < 2; ++sw) {
      launch64_rbgs(ctx->st, U[l], B[l], h2, 0, per, gam(l));
      launch64_rbgs(ctx->st, U[l], B[l], h2, 1, per, gam(l));
    }
  };
  double h2 = 1.0;
  for (int l = 0; l < L; ++l) {
    smooth(l, h2);
    launch64_resid_restrict(ctx->st, U[l], B[l], 1.0 / h2, U[l + 1], B[l + 1], per, gam(l));
    h2 *= 4.0;
  }
  launch64_bottom(ctx->st, U[L], B[L], h2, per, gam(L), 64);
  for (int l = L - 1; l >= 0; --l) {
    h2 *= 0.25;
    launch64_prolong(ctx->st, U[l + 1], U[l], per, gam(l + 1));
    smooth(l, h2);
  }
  CKL();
  return PM_OK;
}

// The solve with the potential, the source and every level in double
// (PM_FP64_PLAIN): Phi (with its ghost layer, the open boundary's Dirichlet
// values) and f widened from their double-float pairs, V-cycles on Phi
// until ||f - A Phi|| / ||f|| <= rtol (read after each), Phi narrowed back
// to a pair for the gradient and the next warm start.
pm_status solve64(pm_ctx* ctx) {
  const int lo = ctx->lo, s = ctx->s, per = ctx->periodic;
  Grid fh = full_view(ctx, ctx->f_hi, lo, s), fl = full_view(ctx, ctx->f_lo, lo, s);
  Grid ph = full_view(ctx, ctx->phi_h[ctx->cur], lo, s);
  Grid pl = full_view(ctx, ctx->phi_l[ctx->cur], lo, s);
  GridD P = full_view64(ctx, ctx->phi64, lo, s), F = full_view64(ctx, ctx->f64, lo, s);
  if (ctx->cfg.guess == PM_GUESS_ZERO) {
    launch_fill(ctx->st, ph, 0.0f, false);
    launch_fill(ctx->st, pl, 0.0f, false);
  }
  launch64_from_pair(ctx->st, ph, pl, P, true);
  launch64_from_pair(ctx->st, fh, fl, F, false);
  ctx->guess_used_last = 0;
  int it = 0;
  double rel = 0.0;
  for (;;) {
    launch64_defect(ctx->st, P, F, per, ctx->partial, ctx->counter, ctx->d_scal + 11);
    CKL();
    pm_status st = sync_read(ctx);
    if (st != PM_OK) return st;
    const double f2 = ctx->h_scal[0], r2 = ctx->h_scal[11];
    rel = f2 > 0 ? std::sqrt(r2 / f2) : 0.0;
    if (it == 0) ctx->resid_start = ctx->resid_guess = rel;
    if (rel <= ctx->cfg.rtol || f2 == 0.0) break;
    if (it >= ctx->cfg.max_vcycles) {
      ctx->vcycles_last = it;
      ctx->vcycles_total += it;
      ctx->resid_last = rel;
      char buf[160];
      snprintf(buf, sizeof buf, "solve: relative residual %.3e after %d V-cycles (rtol %.1e)",
               rel, it, ctx->cfg.rtol);
      return fail(ctx, PM_ENOCONV, buf);
    }
    st = vcycle64(ctx, P, F);
    if (st != PM_OK) return st;
    ++it;
  }
  launch64_to_pair(ctx->st, P, ph, pl, false);
  CKL();
  ctx->vcycles_last = it;
  ctx->vcycles_total += it;
  ctx->resid_last = rel;
  ctx->vc_prev = it;
  return PM_OK;
}

// PM_MIXED_FP64: FP32 V-cycles inside an FP64 defect correction.  The
// potential is FP64 throughout; each iteration adds the last V-cycle's
// correction to it in FP64 (k64_correct), evaluates r = f - A Phi in FP64
// (k64m_defect, r rounded to FP32 as the next V-cycle's right-hand side) and
// its norm; the residual is read on the host as in solve().
pm_status solve_m64(pm_ctx* ctx) {
  const int lo = ctx->lo, s = ctx->s, per = ctx->periodic;
  Grid fh = full_view(ctx, ctx->f_hi, lo, s), fl = full_view(ctx, ctx->f_lo, lo, s);
  Grid e0 = compact_view(ctx->ecorr, s), r0 = compact_view(ctx->lb[0], s);
  GridD P = full_view64(ctx, ctx->phi64, lo, s), F = full_view64(ctx, ctx->f64, lo, s);
  const double cells = (double)s * s * s;
  int e = prof_begin(ctx);
  if (ctx->cfg.guess == PM_GUESS_ZERO) launch64_fill(ctx->st, P, 0.0);
  // the source of this solve in FP64 (hi + lo of the source kernel's pair):
  // reads 8 B and writes 8 B per cell
  launch64_from_pair(ctx->st, fh, fl, F, false);
  prof_end(ctx, PM_PROF_CORRECT, e, 16.0 * cells);
  ctx->guess_used_last = 0;
  int it = 0;
  bool first = true, started = false;
  double rel = 0.0;
  const int blind = std::min(std::max(0, ctx->vc_prev - 1), ctx->cfg.max_vcycles - 1);
  const int inner = std::max(1, ctx->cfg.inner_vcycles);
  for (;;) {
    const int slot = first ? 13 : 11;
    e = prof_begin(ctx);
    // Phi += e: reads Phi (8 B) and e (4), writes Phi (8); the defect reads
    // Phi (8) and f (8) and writes r (4)
    if (!first) launch64_correct(ctx->st, P, e0);
    launch64m_defect(ctx->st, P, F, r0, per, ctx->partial, ctx->counter, ctx->d_scal + slot);
    prof_end(ctx, PM_PROF_DEFECT, e, (first ? 20.0 : 40.0) * cells);
    first = false;
    CKL();
    if (it < blind) {
      // up to `inner` FP32 V-cycles on A e = r before the next FP64 defect
      const int m = std::min(inner, blind - it);
      for (int q = 0; q < m; ++q) {
        pm_status v = vcycle_run(ctx, e0, r0, q == 0);
        if (v != PM_OK) return v;
        ++it;
      }
      continue;
    }
    pm_status st = sync_read(ctx);
    if (st != PM_OK) return st;
    const double f2 = ctx->h_scal[0], r2 = ctx->h_scal[slot];
    rel = f2 > 0 ? std::sqrt(r2 / f2) : 0.0;
    if (!started) {
      started = true;
      ctx->resid_start = f2 > 0 ? std::sqrt(ctx->h_scal[13] / f2) : 0.0;
      ctx->resid_guess = ctx->resid_start;
    }
    if (rel <= ctx->cfg.rtol || f2 == 0.0) break;
    if (it >= ctx->cfg.max_vcycles) {
      ctx->vcycles_last = it;
      ctx->vcycles_total += it;
      ctx->resid_last = rel;
      char buf[160];
      snprintf(buf, sizeof buf, "solve: relative residual %.3e after %d V-cycles (rtol %.1e)",
               rel, it, ctx->cfg.rtol);
      return fail(ctx, PM_ENOCONV, buf);
    }
    pm_status v = vcycle_run(ctx, e0, r0, true);
    if (v != PM_OK) return v;
    ++it;
  }
  ctx->vcycles_last = it;
  ctx->vcycles_total += it;
  ctx->resid_last = rel;
  ctx->vc_prev = it;
  return PM_OK;
}

// The FP64 potential of PM_MIXED_FP64 (current and previous solution, with
// the ghost layer) to / from the double-float pairs that pm_potential's
// setup and outputs use.
void m64_to_pairs(pm_ctx* ctx, int lo, int s) {
  launch64_to_pair(ctx->st, full_view64(ctx, ctx->phi64, lo, s),
                   full_view(ctx, ctx->phi_h[ctx->cur], lo, s),
                   full_view(ctx, ctx->phi_l[ctx->cur], lo, s), true);
}
void m64_from_pairs(pm_ctx* ctx, int lo, int s) {
  launch64_from_pair(ctx->st, full_view(ctx, ctx->phi_h[ctx->cur], lo, s),
                     full_view(ctx, ctx->phi_l[ctx->cur], lo, s),
                     full_view64(ctx, ctx->phi64, lo, s), true);
}

pm_status solve(pm_ctx* ctx) {
  NvtxRange nvtx("pm solve");
  if (ctx->cfg.precision == PM_FP64_PLAIN) return solve64(ctx);
  if (ctx->cfg.precision == PM_MIXED_FP64) return solve_m64(ctx);
  const int lo = ctx->lo, s = ctx->s, per = ctx->periodic;
  Grid fh = full_view(ctx, ctx->f_hi, lo, s), fl = full_view(ctx, ctx->f_lo, lo, s);
  const bool mixed = ctx->cfg.precision == PM_MIXED;
  Grid e0 = compact_view(mixed ? ctx->ecorr : ctx->lu[0], s), r0 = compact_view(ctx->lb[0], s);
  // (the ball solve's defect leaves the cells outside its mask out)
  auto ph_of = [&](int q) { return masked(ctx, full_view(ctx, ctx->phi_h[q], lo, s), 0); };
  auto pl_of = [&](int q) { return full_view(ctx, ctx->phi_l[q], lo, s); };
  if (ctx->cfg.guess == PM_GUESS_ZERO) {
    launch_fill(ctx->st, ph_of(ctx->cur), 0.0f, false);
    launch_fill(ctx->st, pl_of(ctx->cur), 0.0f, false);
  }
  bool net_todo = ctx->cfg.guess == PM_GUESS_LEARNED && guess_fits(ctx->net, s);
  const bool capture = mixed && ctx->cap_r != nullptr;
  ctx->guess_used_last = 0;
  int it = 0;            // V-cycles run
  bool pending = false;  // e0 holds a correction not yet added to Phi
  bool first = true;
  bool started = false;  // the start residual has been read
  int slot = 11;         // d_scal slot of the latest defect's ||r||^2 (13: the first)
  double rel = 0.0;
  const double cells = (double)s * s * s;
  // V-cycles run back to back before the residual is first read on the host:
  // one fewer than the previous solve took (consecutive solves need similar
  // counts), so the GPU does not wait for a host round trip after each; the
  // network start and the pair capture read every residual.
  const int blind = (net_todo || capture)
                        ? 0
                        : std::min(std::max(0, ctx->vc_prev - 1), ctx->cfg.max_vcycles - 1);
  const int inner = std::max(1, ctx->cfg.inner_vcycles);
  for (;;) {
    const int c0 = ctx->cur;
    slot = first ? 13 : 11;
    // the plain path's residual norm is only needed where it is read: at the
    // start (resid_start) and once the blind V-cycles are done
    if (!mixed && !net_todo && !first && it < blind) {
      pm_status v = vcycle_run(ctx, ph_of(ctx->cur), fh, false);
      if (v != PM_OK) return v;
      ++it;
      continue;
    }
    int e = prof_begin(ctx);
    if (mixed && pending) {
      // Phi <- Phi + e, written to the other buffer; reads Phi (8 B), e (4),
      // f (8), writes Phi (8) and r (4) per cell
      if (capture) launch_to_dense(ctx->st, e0, ctx->cap_e, true);
      launch_defect(ctx->st, ph_of(c0), pl_of(c0), &e0, ph_of(c0 ^ 1), pl_of(c0 ^ 1), fh, fl,
                    r0, per, true, ctx->partial, ctx->counter, ctx->d_scal + slot,
                    6.0 + ctx->sig_d);
      ctx->cur ^= 1;
      prof_end(ctx, PM_PROF_DEFECT, e, 32.0 * cells);
    } else {
      launch_defect(ctx->st, ph_of(c0), pl_of(c0), nullptr, ph_of(c0), pl_of(c0), fh, fl, r0,
                    per, mixed || net_todo, ctx->partial, ctx->counter, ctx->d_scal + slot,
                    6.0 + ctx->sig_d);
      prof_end(ctx, PM_PROF_DEFECT, e, (mixed ? 20.0 : 16.0) * cells);
    }
    pending = false;
    if (first && capture) {
      launch_to_dense(ctx->st, r0, ctx->cap_r, false);
      CK(cudaMemsetAsync(ctx->cap_e, 0, sizeof(float) * (size_t)cells, ctx->st));
    }
    first = false;
    CKL();
    if (it < blind) {
      if (mixed) {
        // up to `inner` FP32 V-cycles on the same correction equation
        // A e = r (the first from zero, the next from the iterate; the
        // V-cycle's own FP32 residual drives them) before the next defect
        const int m = std::min(inner, blind - it);
        for (int q = 0; q < m; ++q) {
          pm_status v = vcycle_run(ctx, e0, r0, q == 0);
          if (v != PM_OK) return v;
          ++it;
        }
        pending = true;
      } else {
        pm_status v = vcycle_run(ctx, ph_of(ctx->cur), fh, false);
        if (v != PM_OK) return v;
        ++it;
      }
      continue;
    }
    pm_status st = sync_read(ctx);
    if (st != PM_OK) return st;
    double f2 = ctx->h_scal[0], r2 = ctx->h_scal[slot];
    rel = f2 > 0 ? std::sqrt(r2 / f2) : 0.0;
    if (!started) {
      started = true;
      ctx->resid_start = f2 > 0 ? std::sqrt(ctx->h_scal[13] / f2) : 0.0;
      ctx->resid_guess = ctx->resid_start;
    } else if (it == 0) {
      ctx->resid_guess = rel;  // after the network's correction
    }
    if (rel <= ctx->cfg.rtol || f2 == 0.0) break;
    if (it >= ctx->cfg.max_vcycles) {
      ctx->vcycles_last = it;
      ctx->vcycles_total += it;
      ctx->resid_last = rel;
      char buf[160];
      snprintf(buf, sizeof buf, "solve: relative residual %.3e after %d V-cycles (rtol %.1e)",
               rel, it, ctx->cfg.rtol);
      return fail(ctx, PM_ENOCONV, buf);
    }
    if (net_todo) {
      // e ~ A^-1 r from the network; r = f - A Phi of the start
      net_todo = false;
      e = prof_begin(ctx);
      launch_to_dense(ctx->st, r0, ctx->nn_in, false);
      st = guess_apply(ctx->net, ctx->st, ctx->nn_in, s, per, ctx->nn_out);
      if (st != PM_OK) return fail(ctx, st, pm_guess_last_error(ctx->net));
      if (mixed) {
        launch_from_dense(ctx->st, ctx->nn_out, e0, false);
        pending = true;
      } else {
        launch_from_dense(ctx->st, ctx->nn_out, ph_of(ctx->cur), true);
      }
      prof_end(ctx, PM_PROF_GUESS, e, 16.0 * cells);
      CKL();
      ctx->guess_used_last = 1;
      ctx->guess_used_total++;
      continue;
    }
    // the correction e starts at zero in every V-cycle (zero-start sweep)
    pm_status v = mixed ? vcycle_run(ctx, e0, r0, true)
                        : vcycle_run(ctx, ph_of(ctx->cur), fh, false);
    if (v != PM_OK) return v;
    ++it;
    pending = mixed;
  }
  if (ctx->guess_used_last) {
    pm_status st = guess_check(ctx->net, ctx->st);
    if (st != PM_OK) return fail(ctx, st, "learned guess: an MMA completion wait timed out");
  }
  ctx->vcycles_last = it;
  ctx->vcycles_total += it;
  ctx->resid_last = rel;
  ctx->vc_prev = it;
  return PM_OK;
}

pm_status shrink_to(pm_ctx* ctx, double R, double a_cross, bool flags_ready) {
  NvtxRange nvtx("pm shrink");
  const double c = 0.5 * ctx->n;
  float klo, khi;
  keep_bounds(c, R, &klo, &khi);
  const long long N = ctx->n_active;
  if (N == 0) return PM_OK;
  const int nblk = gkd_blocks(N);
  int e = prof_begin(ctx);
  if (!flags_ready)
    launch_flag(ctx->st, ctx->pos, N, klo, khi, ctx->flags, ctx->block_keep, keep_ball(ctx, R));
  launch_scan_blocks(ctx->st, ctx->block_keep, ctx->keep_off, nblk, ctx->d_cnt);
  launch_scatter(ctx->st, ctx->pos, ctx->mom, N, ctx->flags, ctx->keep_off, ctx->pos2,
                 ctx->mom2, ctx->lc_pos, ctx->lc_mom, ctx->n_lc, (float)a_cross);
  // scatter: read the flag (1 B) and both records (32 B), write them (32 B)
  prof_end(ctx, PM_PROF_COMPACT, e, 65.0 * N);
  CKL();
  pm_status st = sync_read(ctx);
  if (st != PM_OK) return st;
  long long keep = (long long)ctx->h_cnt[0];
  std::swap(ctx->pos, ctx->pos2);
  std::swap(ctx->mom, ctx->mom2);
  ctx->n_lc += N - keep;
  ctx->n_active = keep;
  return PM_OK;
}

// Fixed-box lightcone record: copy the active particles that lie outside the
// keep cube of radius R and carry no record mark into the lightcone buffer
// (index order), marking them; nobody leaves the active set.
pm_status record_to(pm_ctx* ctx, double R, double a_cross) {
  float klo, khi;
  keep_bounds(0.5 * ctx->n, R, &klo, &khi);
  const long long N = ctx->n_active;
  if (N == 0) return PM_OK;
  const int nblk = gkd_blocks(N);
  int e = prof_begin(ctx);
  launch_flag_record(ctx->st, ctx->pos, ctx->mom, N, klo, khi, ctx->flags, ctx->block_keep,
                     keep_ball(ctx, R));
  launch_scan_blocks(ctx->st, ctx->block_keep, ctx->keep_off, nblk, ctx->d_cnt);
  launch_record(ctx->st, ctx->pos, ctx->mom, N, ctx->flags, ctx->keep_off, ctx->lc_pos,
                ctx->lc_mom, ctx->n_lc, ctx->N0, (float)a_cross);
  // read both records and the flag (33 B), write the recorded ones
  prof_end(ctx, PM_PROF_COMPACT, e, 33.0 * N);
  CKL();
  pm_status st = sync_read(ctx);
  if (st != PM_OK) return st;
  const long long rec = (long long)ctx->h_cnt[0];
  if (ctx->n_lc + rec > ctx->N0)
    return fail(ctx, PM_EOVERFLOW, "lightcone record: more records than particles (a set "
                                   "of particles without cleared record marks?)");
  ctx->n_lc += rec;
  return PM_OK;
}

pm_status alloc(pm_ctx* ctx, void** p, size_t bytes) {
  // host-side fault injection for tests: PM_FAULT_ALLOC=k makes the k-th
  // device allocation of a context fail as if the device were full
  const char* fk = getenv("PM_FAULT_ALLOC");
  if (ctx && fk && ++ctx->n_allocs == atoll(fk)) {
    *p = nullptr;
    return fail(ctx, PM_ENOMEM, "cudaMalloc: allocation failure injected (PM_FAULT_ALLOC)");
  }
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    return fail(ctx, PM_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  return PM_OK;
}

}  // namespace

// Keep rule of pm_shrink for callers outside a context (see noalloc.cu).
double pm::shrink_radius_cells(int n, double box, double om, double ol, double buffer,
                               double a) {
  double chi = C_OVER_H0 * (tau_of_a(1.0, om, ol) - tau_of_a(a, om, ol));
  return chi / (box / n) + buffer;
}

void pm::shrink_keep_bounds(int n, double R, float* klo, float* khi) {
  if (R <= 0.5 * n - 1.0) {
    keep_bounds(0.5 * n, R, klo, khi);
  } else {  // periodic phase under PM_BC_PAPER: nothing leaves
    *klo = -3.402823466e38f;
    *khi = 3.402823466e38f;
  }
}

extern "C" {

void pm_config_default(pm_config* c) {
  std::memset(c, 0, sizeof(*c));
  c->n_mesh = 32;
  c->n_particles = 32 * 32 * 32;
  c->box_mpch = 250.0;
  c->omega_m = 0.3;
  c->omega_l = 0.7;
  c->a_init = 0.02;
  c->a_final = 1.0;
  c->n_steps = 20;
  c->rtol = 1e-7;
  c->max_vcycles = 50;
  c->precision = PM_MIXED;
  c->guess = PM_GUESS_WARM;
  c->bc = PM_BC_PAPER;
  c->shrink = 1;
  c->buffer_cells = 1.0;
  c->store_forces = 0;
  c->inner_vcycles = 1;
  c->gravity = PM_GRAVITY_POISSON;
  c->c_eff_factor = 0.019;
  c->assignment = PM_ASSIGN_CIC;
  c->domain = PM_DOMAIN_CUBE;
}

pm_status pm_init(const pm_config* cfg, const float* pos4, const float* mom4,
                  int32_t host_mem, void* stream, pm_ctx** out) {
  pm_ctx* ctx = nullptr;
  if (!out) return fail(nullptr, PM_EINVAL, "pm_init: out is NULL");
  *out = nullptr;
  if (!cfg || !pos4 || !mom4) return fail(nullptr, PM_EINVAL, "pm_init: NULL argument");
  if (!mg_size_ok(cfg->n_mesh) || cfg->n_mesh > 1024)
    return fail(nullptr, PM_EINVAL, "pm_init: n_mesh must be 2^j or 3*2^j in [4, 1024]");
  if (cfg->n_particles <= 0 || cfg->n_particles >= (1LL << 31))
    return fail(nullptr, PM_EINVAL, "pm_init: n_particles must be in [1, 2^31)");
  // omega_m >= 1e-6: the conformal-time quadrature (64 Gauss panels in
  // u = sqrt(a)) resolves the peak of width (omega_m / omega_l)^(1/6) at u = 0
  if (cfg->n_steps <= 0 || !(cfg->a_init > 0) || !(cfg->a_final > cfg->a_init) ||
      !(cfg->box_mpch > 0) || !(cfg->omega_m >= 1e-6) || cfg->omega_l < 0 ||
      !(cfg->rtol > 0) ||
      cfg->max_vcycles < 1)
    return fail(nullptr, PM_EINVAL, "pm_init: invalid schedule, cosmology or tolerance");
  if (cfg->precision != PM_MIXED && cfg->precision != PM_FP32_PLAIN &&
      cfg->precision != PM_FP64_PLAIN && cfg->precision != PM_MIXED_FP64)
    return fail(nullptr, PM_EINVAL, "pm_init: unknown precision");
  if (cfg->precision == PM_MIXED_FP64 &&
      (cfg->gravity != PM_GRAVITY_POISSON || cfg->guess == PM_GUESS_LEARNED))
    return fail(nullptr, PM_EINVAL, "pm_init: PM_MIXED_FP64 solves Poisson's equation from "
                                    "the warm or zero start");
  if (cfg->precision == PM_FP64_PLAIN &&
      (cfg->gravity != PM_GRAVITY_POISSON || cfg->guess == PM_GUESS_LEARNED))
    return fail(nullptr, PM_EINVAL, "pm_init: PM_FP64_PLAIN solves Poisson's equation from "
                                    "the warm or zero start");
  if (cfg->bc < PM_BC_PAPER || cfg->bc > PM_BC_PERIODIC)
    return fail(nullptr, PM_EINVAL, "pm_init: unknown bc");
  if (cfg->guess < PM_GUESS_WARM || cfg->guess > PM_GUESS_LEARNED)
    return fail(nullptr, PM_EINVAL, "pm_init: unknown guess");
  if (cfg->shrink < PM_SHRINK_OFF || cfg->shrink > PM_SHRINK_RECORD)
    return fail(nullptr, PM_EINVAL, "pm_init: unknown shrink mode");
  if (cfg->domain != PM_DOMAIN_CUBE &&
      ((cfg->domain != PM_DOMAIN_SPHERE && cfg->domain != PM_DOMAIN_BALL) ||
       cfg->assignment != PM_ASSIGN_CIC))
    return fail(nullptr, PM_EINVAL, "pm_init: domain is the cube, or the sphere or ball with CIC");
  if (cfg->domain == PM_DOMAIN_BALL &&
      (cfg->precision != PM_MIXED || cfg->gravity != PM_GRAVITY_POISSON ||
       cfg->guess == PM_GUESS_LEARNED))
    return fail(nullptr, PM_EINVAL, "pm_init: the ball solve needs PM_MIXED, Poisson gravity "
                                    "and the warm or zero start");
  if (cfg->assignment != PM_ASSIGN_CIC &&
      (cfg->assignment != PM_ASSIGN_TSC || cfg->gravity != PM_GRAVITY_POISSON))
    return fail(nullptr, PM_EINVAL, "pm_init: assignment is CIC, or TSC with Poisson gravity");
  if (cfg->sort_every < 0)
    return fail(nullptr, PM_EINVAL, "pm_init: sort_every must be >= 0");
  if (cfg->inner_vcycles < 0 || cfg->inner_vcycles > 16)
    return fail(nullptr, PM_EINVAL, "pm_init: inner_vcycles must be in [0, 16]");
  if (cfg->gravity != PM_GRAVITY_POISSON &&
      ((cfg->gravity != PM_GRAVITY_DIFFUSION && cfg->gravity != PM_GRAVITY_DIFFUSION_ADE) ||
       !(cfg->c_eff_factor > 0) || cfg->precision != PM_MIXED ||
       cfg->guess == PM_GUESS_LEARNED))
    return fail(nullptr, PM_EINVAL,
                "pm_init: diffusion gravity needs c_eff_factor > 0, PM_MIXED, no learned guess");

  if (mg_prepare() != cudaSuccess)
    return fail(nullptr, PM_ECUDA, "pm_init: setting kernel attributes failed");
  ctx = new pm_ctx();
  ctx->cfg = *cfg;
  ctx->st = (cudaStream_t)stream;
  ctx->use_graphs = stream != nullptr && getenv("PM_NO_GRAPHS") == nullptr;
  ctx->n = cfg->n_mesh;
  ctx->P = cfg->n_mesh + 2;
  ctx->N0 = cfg->n_particles;

  // schedule (steps uniform in a, Sec. 3)
  const int K = cfg->n_steps;
  const double om = cfg->omega_m, ol = cfg->omega_l;
  const double cell = cfg->box_mpch / cfg->n_mesh;
  ctx->a.resize(K + 1);
  ctx->dtau.assign(K + 1, 0.0);
  ctx->a_half.assign(K + 1, 0.0);
  ctx->chi.resize(K + 1);
  ctx->R.resize(K + 1);
  std::vector<double> t(K + 1);
  const double t1 = tau_of_a(1.0, om, ol);
  for (int k = 0; k <= K; ++k) {
    ctx->a[k] = cfg->a_init + (cfg->a_final - cfg->a_init) * k / K;
    t[k] = tau_of_a(ctx->a[k], om, ol);
    ctx->chi[k] = C_OVER_H0 * (t1 - t[k]);
    ctx->R[k] = ctx->chi[k] / cell + cfg->buffer_cells;
  }
  for (int k = 0; k < K; ++k) {
    ctx->dtau[k] = t[k + 1] - t[k];
    ctx->a_half[k] = a_of_tau(t[k] + 0.5 * ctx->dtau[k], om, ol);
  }

  const int n = ctx->n, P = ctx->P;
  const long long N = ctx->N0;
  const size_t padded = (size_t)P * P * P;
  pm_status st = PM_OK;
#define AL(ptr, bytes)                                           \
  do {                                                           \
    st = alloc(ctx, (void**)&(ptr), (bytes));                    \
    if (st != PM_OK) { g_err = ctx->err; pm_destroy(ctx); return st; } \
  } while (0)
  AL(ctx->pos, sizeof(float4) * N);
  AL(ctx->mom, sizeof(float4) * N);
  AL(ctx->pos2, sizeof(float4) * N);
  AL(ctx->mom2, sizeof(float4) * N);
  AL(ctx->lc_pos, sizeof(float4) * N);
  AL(ctx->lc_mom, sizeof(float4) * N);
  if (cfg->store_forces) AL(ctx->forces, sizeof(float4) * N);
  AL(ctx->flags, N);
  const int nblk = gkd_blocks(N);
  AL(ctx->block_keep, sizeof(unsigned int) * nblk);
  AL(ctx->keep_off, sizeof(unsigned long long) * nblk);
  AL(ctx->rho, sizeof(unsigned long long) * (size_t)n * n * n);
  for (int q = 0; q < 2; ++q) {
    AL(ctx->phi_h[q], sizeof(float) * padded);
    AL(ctx->phi_l[q], sizeof(float) * padded);
  }
  AL(ctx->grad, sizeof(float4) * padded);
  AL(ctx->f_hi, sizeof(float) * padded);
  AL(ctx->f_lo, sizeof(float) * padded);
  AL(ctx->prev_hi, sizeof(float) * padded);
  AL(ctx->prev_lo, sizeof(float) * padded);
  for (int sl = n;; sl /= 2) {
    float *u = nullptr, *b = nullptr;
    size_t bytes = sizeof(float) * (size_t)(sl + 2) * (sl + 2) * (sl + 2);
    AL(u, bytes);
    ctx->lu.push_back(u);
    AL(b, bytes);
    ctx->lb.push_back(b);
    float* u2 = nullptr;
    AL(u2, bytes);
    ctx->lu2.push_back(u2);
    if (cfg->precision == PM_FP64_PLAIN) {
      double *u64 = nullptr, *b64 = nullptr;
      if (ctx->lu.size() > 1) {  // level 0 is the full grid
        AL(u64, 2 * bytes);
        AL(b64, 2 * bytes);
      }
      ctx->lu64.push_back(u64);
      ctx->lb64.push_back(b64);
    }
    if (sl <= 4 || sl % 2) break;
  }
  if (cfg->precision == PM_FP64_PLAIN || cfg->precision == PM_MIXED_FP64) {
    AL(ctx->phi64, sizeof(double) * padded);
    AL(ctx->f64, sizeof(double) * padded);
  }
  if (cfg->precision == PM_MIXED_FP64) AL(ctx->prev64, sizeof(double) * padded);
  if (cfg->precision == PM_MIXED || cfg->precision == PM_MIXED_FP64)
    AL(ctx->ecorr, sizeof(float) * padded);
  const int maxblk = std::max(std::max(SRC_GRID, defect_blocks(n)), 4096);
  AL(ctx->partial, sizeof(double) * 16 * maxblk);
  AL(ctx->partial_m, 16 * 10 * (size_t)maxblk);
  AL(ctx->counter, sizeof(unsigned int) * 4);
  AL(ctx->d_scal, sizeof(double) * 16);
  AL(ctx->bgm, BGW_OFF + sizeof(df) * (size_t)n);
  ctx->bgw = (df*)((char*)ctx->bgm + BGW_OFF);
  if (cfg->domain != PM_DOMAIN_CUBE) {
    AL(ctx->ballw, sizeof(float) * (size_t)n * n * n);
    ctx->ball_rule = ball_rule();
  }
  if (cfg->sort_every > 0) {
    for (int q = 0; q < 2; ++q) {
      AL(ctx->sortw.keys[q], sizeof(unsigned) * N);
      AL(ctx->sortw.vals[q], sizeof(unsigned) * N);
    }
    AL(ctx->sortw.counts, sizeof(unsigned) * sort_counts_len(N));
    AL(ctx->sortw.ghist, sizeof(unsigned) * sort_ghist_len());
  }
  ctx->h_bg.assign(BGW_OFF + sizeof(df) * (size_t)n, 0);
  AL(ctx->d_cnt, sizeof(unsigned long long) * 4);
  ctx->d_overflow = (int*)(ctx->d_cnt + 3);  // read back with every sync_read
#undef AL
  if (cudaMallocHost((void**)&ctx->h_scal, sizeof(double) * 16) != cudaSuccess ||
      cudaMallocHost((void**)&ctx->h_cnt, sizeof(unsigned long long) * 4) != cudaSuccess) {
    g_err = "pm_init: cudaMallocHost failed";
    pm_destroy(ctx);
    return PM_ENOMEM;
  }
  cudaStream_t s0 = ctx->st;
#define Z(ptr, bytes)                                                        \
  if (cudaMemsetAsync((ptr), 0, (bytes), s0) != cudaSuccess) {               \
    g_err = "pm_init: cudaMemsetAsync failed"; pm_destroy(ctx); return PM_ECUDA; }
  Z(ctx->rho, sizeof(unsigned long long) * (size_t)n * n * n);
  Z(ctx->phi_h[0], sizeof(float) * padded);
  Z(ctx->phi_l[0], sizeof(float) * padded);
  Z(ctx->phi_h[1], sizeof(float) * padded);
  Z(ctx->phi_l[1], sizeof(float) * padded);
  Z(ctx->f_hi, sizeof(float) * padded);
  Z(ctx->f_lo, sizeof(float) * padded);
  Z(ctx->prev_hi, sizeof(float) * padded);
  Z(ctx->prev_lo, sizeof(float) * padded);
  if (ctx->phi64) Z(ctx->phi64, sizeof(double) * padded);
  if (ctx->prev64) Z(ctx->prev64, sizeof(double) * padded);
  if (ctx->ecorr) Z(ctx->ecorr, sizeof(float) * padded);
  Z(ctx->counter, sizeof(unsigned int) * 4);
  Z(ctx->d_scal, sizeof(double) * 16);
  Z(ctx->d_cnt, sizeof(unsigned long long) * 4);
#undef Z
  if (tune_fused(ctx) != cudaSuccess) {
    g_err = "pm_init: timing the fused smoother failed";
    pm_destroy(ctx);
    return PM_ECUDA;
  }
  cudaMemcpyKind kind = host_mem ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  if (cudaMemcpyAsync(ctx->pos, pos4, sizeof(float4) * N, kind, s0) != cudaSuccess ||
      cudaMemcpyAsync(ctx->mom, mom4, sizeof(float4) * N, kind, s0) != cudaSuccess ||
      (cfg->shrink == PM_SHRINK_RECORD &&
       cudaMemset2DAsync((char*)ctx->mom + 3 * sizeof(float), sizeof(float4), 0, sizeof(float),
                         (size_t)N, s0) != cudaSuccess) ||
      cudaStreamSynchronize(s0) != cudaSuccess) {
    g_err = "pm_init: copying particles failed";
    pm_destroy(ctx);
    return PM_ECUDA;
  }
  ctx->n_active = N;
  *out = ctx;
  return PM_OK;
}

pm_status pm_step(pm_ctx* ctx, int32_t n_steps) {
  if (!ctx) return fail(nullptr, PM_EINVAL, "pm_step: NULL context");
  if (n_steps < 0 || ctx->step + n_steps > ctx->cfg.n_steps)
    return fail(ctx, PM_EINVAL, "pm_step: past the last step of the schedule");
  if (ctx->cfg.guess == PM_GUESS_LEARNED && !ctx->net)
    return fail(ctx, PM_EINVAL, "pm_step: PM_GUESS_LEARNED without a network (pm_set_guess)");
  const int n = ctx->n;
  const bool mixed = ctx->cfg.precision == PM_MIXED;
  const bool m64 = ctx->cfg.precision == PM_MIXED_FP64;  // Phi kept in FP64
  const bool pair = ctx->cfg.precision != PM_FP32_PLAIN;  // Phi kept as hi + lo
  for (int q = 0; q < n_steps; ++q) {
    NvtxRange nvtx_step("pm step");
    const int k = ctx->step;
    const double R0 = ctx->R[k], R1 = ctx->R[k + 1];
    int lo, s, per;
    geometry(ctx, R0, &lo, &s, &per);
    const bool set_phase_changed = !ctx->cube_valid || per != ctx->periodic;
    pm_status st = set_cube(ctx, lo, s, per, R0);
    if (st != PM_OK) return st;
    const long long N = ctx->n_active;
    if (ctx->cfg.sort_every > 0 && k % ctx->cfg.sort_every == 0 && N > 1) {
      // particle order by cell: keys (read x 16 B, write key + index 8 B),
      // per pass a histogram (4 B) and a scatter (read and write key + index,
      // 16 B), then the permutation (4 B) and both records (read and write,
      // 64 B)
      NvtxRange nvtx_sort("pm sort");
      int es = prof_begin(ctx);
      CK(launch_sort_particles(ctx->st, ctx->pos, ctx->mom, N, n, ctx->sortw, ctx->pos2,
                               ctx->mom2));
      prof_end(ctx, PM_PROF_SORT, es, (24.0 + 20.0 * sort_passes(n) + 68.0) * N);
      std::swap(ctx->pos, ctx->pos2);
      std::swap(ctx->mom, ctx->mom2);
    }
    const double cells = (double)s * s * s;
    const bool diffusion = ctx->cfg.gravity != PM_GRAVITY_POISSON;
    const bool ade = ctx->cfg.gravity == PM_GRAVITY_DIFFUSION_ADE;
    const double nbar = (double)ctx->N0 / ((double)n * n * n);
    const double invM = 1.0 / (281474976710656.0 * nbar);
    Grid fh = full_view(ctx, ctx->f_hi, lo, s), fl = full_view(ctx, ctx->f_lo, lo, s);
    // boundary values of the current source (moments in d_scal) with factor S
    auto ghosts = [&](double Sb) {
      if (per) return;
      int eb = prof_begin(ctx);
      // both buffers carry the ghosts
      const Grid h2 = full_view(ctx, ctx->phi_h[ctx->cur ^ 1], lo, s);
      const Grid l2 = full_view(ctx, ctx->phi_l[ctx->cur ^ 1], lo, s);
      launch_boundary(ctx->st, full_view(ctx, ctx->phi_h[ctx->cur], lo, s),
                      full_view(ctx, ctx->phi_l[ctx->cur], lo, s), n, lo, ctx->d_scal + 1, Sb,
                      true, &h2, &l2);
      prof_end(ctx, PM_PROF_BOUNDARY, eb, 8.0 * 6.0 * (s + 2.0) * (s + 2.0));
    };
    if (diffusion && !ctx->field_ready) {
      // the field starts from the static solution for the initial density
      const double S0 = 1.5 * ctx->cfg.omega_m / ctx->a[k];
      launch_drift_deposit(ctx->st, std::max(1, std::min(gkd_blocks(N) * 4, 152 * 16)),
                           ctx->pos, ctx->mom, N, 0.0f, false, n, lo, s, per, ctx->rho,
                           ctx->d_cnt + 1);
      launch_source(ctx->st, SRC_GRID, ctx->rho, n, lo, s, fh, fl, invM, S0, ctx->bgw,
                    per ? nullptr : ctx->ballw, !per,
                    ctx->partial, ctx->partial_m, ctx->counter, ctx->d_scal, ctx->bgm,
                    ctx->d_overflow);
      ghosts(S0);
      for (int q = 0; q < 2; ++q) {
        launch_fill(ctx->st, full_view(ctx, ctx->phi_h[q], lo, s), 0.0f, false);
        launch_fill(ctx->st, full_view(ctx, ctx->phi_l[q], lo, s), 0.0f, false);
      }
      ctx->sig = 0.0f;
      ctx->sig_d = 0.0;
      CKL();
      st = solve(ctx);
      if (st != PM_OK) return st;
      ctx->field_ready = true;
    }
    // 1-2. half drift + CIC deposit: read x, p, write x (48 B/particle); the
    // count grid is read and written once (16 B/cell)
    int e = prof_begin(ctx);
    if (ctx->cfg.assignment == PM_ASSIGN_TSC)
      launch_drift_deposit_tsc(ctx->st, N, ctx->pos, ctx->mom,
                               (float)(ctx->dtau[k] / (2.0 * ctx->a[k])), true, n, lo, s, per,
                               ctx->rho, ctx->d_cnt + 1);
    else
      launch_drift_deposit(ctx->st, std::max(1, std::min(gkd_blocks(N) * 4, 152 * 16)),
                           ctx->pos, ctx->mom, N, (float)(ctx->dtau[k] / (2.0 * ctx->a[k])),
                           true, n, lo, s, per, ctx->rho, ctx->d_cnt + 1);
    prof_end(ctx, PM_PROF_DEPOSIT, e, 48.0 * N + 16.0 * cells);
    // 3. source, boundary values, solve
    const double S = 1.5 * ctx->cfg.omega_m / ctx->a_half[k];
    e = prof_begin(ctx);
    launch_source(ctx->st, SRC_GRID, ctx->rho, n, lo, s, fh, fl, invM, S, ctx->bgw,
                  per ? nullptr : ctx->ballw, !per,
                  ctx->partial, ctx->partial_m, ctx->counter, ctx->d_scal, ctx->bgm,
                  ctx->d_overflow);
    // read the counts, clear them, write f hi + lo: 24 B/cell
    prof_end(ctx, PM_PROF_SOURCE, e, 24.0 * cells);
    // diffusion: the shift of a half-substep ending at a_e
    const double c_cells = ctx->cfg.c_eff_factor * C_OVER_H0;
    auto shift = [&](double a_e) {
      const double E = std::sqrt(ctx->cfg.omega_m / (a_e * a_e * a_e) + ctx->cfg.omega_l);
      return 3.0 * a_e * E / (c_cells * c_cells * 0.5 * ctx->dtau[k]);
    };
    auto set_shift = [&](double sg) {
      ctx->sig_d = sg;
      ctx->sig = (float)sg;
    };
    if (ade) {
      // substep 1 (t -> t + dt/2): one upward explicit sweep, in place
      ghosts(S);
      e = prof_begin(ctx);
      CK(launch_ade_sweep(ctx->st, full_view(ctx, ctx->phi_h[ctx->cur], lo, s),
                          full_view(ctx, ctx->phi_l[ctx->cur], lo, s), fh, fl, 1.0, per,
                          1.0 / shift(ctx->a_half[k]), true));
      // read f and Phi (16 B), write Phi (8 B) per cell
      prof_end(ctx, PM_PROF_ADE, e, 24.0 * cells);
      CKL();
    } else if (diffusion) {
      // substep 1 (t -> t + dt/2): g = f - sig Phi_old, f kept for substep 2
      ghosts(S);
      const double sg = shift(ctx->a_half[k]);
      e = prof_begin(ctx);
      launch_diff_rhs(ctx->st, SRC_GRID, fh, fl, 1.0, full_view(ctx, ctx->phi_h[ctx->cur], lo, s),
                      full_view(ctx, ctx->phi_l[ctx->cur], lo, s), sg, fh, fl,
                      full_view(ctx, ctx->prev_hi, lo, s), full_view(ctx, ctx->prev_lo, lo, s),
                      true, ctx->partial, ctx->counter, ctx->d_scal);
      prof_end(ctx, PM_PROF_CORRECT, e, 32.0 * cells);
      set_shift(sg);
      CKL();
    } else if (!per && m64) {
      e = prof_begin(ctx);
      launch_boundary64(ctx->st, full_view64(ctx, ctx->phi64, lo, s), n, lo, ctx->d_scal + 1, S);
      prof_end(ctx, PM_PROF_BOUNDARY, e, 8.0 * 6.0 * (s + 2.0) * (s + 2.0));
    } else if (!per && !ctx->mbase) {
      e = prof_begin(ctx);
      // both buffers carry the ghosts in the mixed form (its defect writes
      // Phi + e to the other buffer)
      const Grid h2 = full_view(ctx, ctx->phi_h[ctx->cur ^ 1], lo, s);
      const Grid l2 = full_view(ctx, ctx->phi_l[ctx->cur ^ 1], lo, s);
      launch_boundary(ctx->st, full_view(ctx, ctx->phi_h[ctx->cur], lo, s),
                      full_view(ctx, ctx->phi_l[ctx->cur], lo, s), n, lo, ctx->d_scal + 1, S,
                      pair, mixed ? &h2 : nullptr, mixed ? &l2 : nullptr);
      prof_end(ctx, PM_PROF_BOUNDARY, e, 8.0 * 6.0 * (s + 2.0) * (s + 2.0));
    }
    CKL();
    // warm start extrapolated linearly in a_half from the last two solutions
    // of the same boundary phase (the diffusion substeps start from Phi_old)
    if (!diffusion &&
        (ctx->cfg.guess == PM_GUESS_WARM || ctx->cfg.guess == PM_GUESS_LEARNED)) {
      if (set_phase_changed) ctx->n_sol = 0;
      if (ctx->n_sol >= 1) {
        float w = 0.0f;
        if (ctx->n_sol >= 2) {
          double d0 = ctx->ah_hist[1] - ctx->ah_hist[0];
          w = d0 > 0 ? (float)((ctx->a_half[k] - ctx->ah_hist[1]) / d0) : 0.0f;
        }
        e = prof_begin(ctx);
        if (m64) {
          double w64 = 0.0;
          if (ctx->n_sol >= 2) {
            double d0 = ctx->ah_hist[1] - ctx->ah_hist[0];
            w64 = d0 > 0 ? (ctx->a_half[k] - ctx->ah_hist[1]) / d0 : 0.0;
          }
          launch64_predict(ctx->st, full_view64(ctx, ctx->phi64, lo, s),
                           full_view64(ctx, ctx->prev64, lo, s), w64);
        } else {
          launch_predict(ctx->st, full_view(ctx, ctx->phi_h[ctx->cur], lo, s),
                         full_view(ctx, ctx->phi_l[ctx->cur], lo, s),
                         full_view(ctx, ctx->prev_hi, lo, s),
                         full_view(ctx, ctx->prev_lo, lo, s), w, pair);
        }
        prof_end(ctx, PM_PROF_CORRECT, e, 32.0 * cells);
      }
    }
    if (ctx->mbase) {
      // the ball solve's Dirichlet values, after the prediction (its ghost
      // cells lie inside the cube, where the prediction extrapolates)
      e = prof_begin(ctx);
      launch_ball_ghosts(ctx->st, masked(ctx, full_view(ctx, ctx->phi_h[ctx->cur], lo, s), 0),
                         full_view(ctx, ctx->phi_l[ctx->cur], lo, s),
                         full_view(ctx, ctx->phi_h[ctx->cur ^ 1], lo, s),
                         full_view(ctx, ctx->phi_l[ctx->cur ^ 1], lo, s), n, lo,
                         ctx->d_scal + 1, S);
      // 16 B per cell outside the ball's mask (about half the cube)
      prof_end(ctx, PM_PROF_BOUNDARY, e, 8.0 * (s + 2.0) * (s + 2.0) * (s + 2.0));
      CKL();
    }
    if (!ade) {
      st = solve(ctx);
      ctx->sig = 0.0f;
      ctx->sig_d = 0.0;
      if (st != PM_OK) return st;
      ctx->ah_hist[0] = ctx->ah_hist[1];
      ctx->ah_hist[1] = ctx->a_half[k];
      ctx->n_sol++;
    }
    // 4-6. gradient + gather + kick + half drift (+ keep flags)
    const bool do_flag =
        ctx->cfg.shrink == PM_SHRINK_ON && ctx->cfg.bc != PM_BC_PERIODIC && is_open(ctx, R1);
    float klo = 0.f, khi = 0.f;
    if (do_flag) keep_bounds(0.5 * n, R1, &klo, &khi);
    e = prof_begin(ctx);
    // gradient field: read Phi hi + lo, write G (24 B/cell)
    if (m64)
      launch64_grad(ctx->st, ctx->phi64, n, lo, s, per, ctx->grad);
    else
      launch_grad(ctx->st, ctx->phi_h[ctx->cur], ctx->phi_l[ctx->cur], n, lo, s, per, ctx->grad);
    if (ctx->cfg.assignment == PM_ASSIGN_TSC)
      launch_gather_tsc(ctx->st, ctx->pos, ctx->mom, N, ctx->grad, n, lo, s, per,
                        (float)(ctx->a_half[k] * ctx->dtau[k]),
                        (float)(ctx->dtau[k] / (2.0 * ctx->a[k + 1])), do_flag, klo, khi,
                        ctx->flags, ctx->block_keep, ctx->forces, ctx->d_cnt + 1);
    else
      launch_gather_kick_drift(ctx->st, ctx->pos, ctx->mom, N, ctx->phi_h[ctx->cur],
                               ctx->phi_l[ctx->cur], ctx->grad, n, lo, s,
                               per, (float)(ctx->a_half[k] * ctx->dtau[k]),
                               (float)(ctx->dtau[k] / (2.0 * ctx->a[k + 1])), do_flag, klo,
                               khi, keep_ball(ctx, R1), ctx->flags, ctx->block_keep,
                               ctx->forces, ctx->d_cnt + 1);
    // gather: read x, p, write x, p (64 B/particle, + 1 B flag), read G once
    // (16 B/cell)
    prof_end(ctx, PM_PROF_GATHER, e, (do_flag ? 65.0 : 64.0) * N + (24.0 + 16.0) * cells);
    CKL();
    ctx->forces_valid = ctx->forces != nullptr;
    ctx->forces_n = N;
    if (ade) {
      // substep 2 (t + dt/2 -> t + dt): the same density, S and H at a_{n+1},
      // one downward sweep
      const double S2 = 1.5 * ctx->cfg.omega_m / ctx->a[k + 1];
      ghosts(S2);
      e = prof_begin(ctx);
      CK(launch_ade_sweep(ctx->st, full_view(ctx, ctx->phi_h[ctx->cur], lo, s),
                          full_view(ctx, ctx->phi_l[ctx->cur], lo, s), fh, fl, S2 / S, per,
                          1.0 / shift(ctx->a[k + 1]), false));
      prof_end(ctx, PM_PROF_ADE, e, 24.0 * cells);
      CKL();
    } else if (diffusion) {
      // substep 2 (t + dt/2 -> t + dt): the same density, S and H at a_{n+1}
      const double S2 = 1.5 * ctx->cfg.omega_m / ctx->a[k + 1];
      ghosts(S2);
      const double sg = shift(ctx->a[k + 1]);
      e = prof_begin(ctx);
      launch_diff_rhs(ctx->st, SRC_GRID, full_view(ctx, ctx->prev_hi, lo, s),
                      full_view(ctx, ctx->prev_lo, lo, s), S2 / S,
                      full_view(ctx, ctx->phi_h[ctx->cur], lo, s),
                      full_view(ctx, ctx->phi_l[ctx->cur], lo, s), sg, fh, fl, fh, fl, false,
                      ctx->partial, ctx->counter, ctx->d_scal);
      prof_end(ctx, PM_PROF_CORRECT, e, 28.0 * cells);
      set_shift(sg);
      CKL();
      st = solve(ctx);
      ctx->sig = 0.0f;
      ctx->sig_d = 0.0;
      if (st != PM_OK) return st;
    }
    // 7. lightcone shrink (or, in the fixed box, the lightcone record)
    if (do_flag) {
      st = shrink_to(ctx, R1, ctx->a[k + 1], true);
      if (st != PM_OK) return st;
    } else if (ctx->cfg.shrink == PM_SHRINK_RECORD && R1 <= 0.5 * n - 1.0) {
      // the keep cube lies inside the box (whatever the solve's boundary)
      st = record_to(ctx, R1, ctx->a[k + 1]);
      if (st != PM_OK) return st;
    }
    // the source kernel flags a cell count above 2^62 in d_cnt[3], which the
    // solve's residual reads bring back; the step itself ends without a
    // host synchronisation (its profile events are flushed at the next read)
    if (ctx->h_cnt[3]) return fail(ctx, PM_EOVERFLOW, "deposit: a cell count exceeded 2^62");
    ctx->particle_steps += N;
    ctx->step++;
  }
  return PM_OK;
}

pm_status pm_shrink(pm_ctx* ctx, double a, int64_t* n_active_out) {
  if (!ctx) return fail(nullptr, PM_EINVAL, "pm_shrink: NULL context");
  if (!(a > 0)) return fail(ctx, PM_EINVAL, "pm_shrink: a must be > 0");
  // the keep rule shared with the allocation-free compaction (noalloc.cu)
  const double R = pm::shrink_radius_cells(ctx->n, ctx->cfg.box_mpch, ctx->cfg.omega_m,
                                           ctx->cfg.omega_l, ctx->cfg.buffer_cells, a);
  if (is_open(ctx, R) && ctx->cfg.bc != PM_BC_PERIODIC) {
    pm_status st = shrink_to(ctx, R, a, false);
    if (st != PM_OK) return st;
  }
  if (n_active_out) *n_active_out = ctx->n_active;
  return PM_OK;
}

pm_status pm_potential(pm_ctx* ctx, const double* delta_dev, double a, int32_t bc,
                       float* phi_out_dev, double* phi64_out_dev, int32_t* vcycles_out,
                       double* resid_out) {
  if (!ctx) return fail(nullptr, PM_EINVAL, "pm_potential: NULL context");
  if (!delta_dev || !phi_out_dev || !(a > 0) || (bc != PM_BC_OPEN && bc != PM_BC_PERIODIC))
    return fail(ctx, PM_EINVAL, "pm_potential: bad argument");
  const int n = ctx->n;
  const int per = bc == PM_BC_PERIODIC;
  pm_status st = set_cube(ctx, 0, n, per, 1e300);
  if (st != PM_OK) return st;
  ctx->cube_valid = false;  // the next step re-derives its cube
  ctx->n_sol = 0;           // and does not extrapolate across this solve
  ctx->field_ready = false; // a diffusion run restarts its field
  const double S = 1.5 * ctx->cfg.omega_m / a;
  Grid fh = full_view(ctx, ctx->f_hi, 0, n), fl = full_view(ctx, ctx->f_lo, 0, n);
  const bool pair = ctx->cfg.precision != PM_FP32_PLAIN;  // Phi kept as hi + lo
  launch_source_f64(ctx->st, SRC_GRID, delta_dev, n, fh, fl, S, !per, ctx->partial,
                    ctx->counter, ctx->d_scal);
  // launch_source_f64 writes (||f||^2, q0, d, S_ab) to d_scal[0..10]
  for (int q = 0; q < 2; ++q) {
    Grid gh = full_view(ctx, ctx->phi_h[q], 0, n), gl = full_view(ctx, ctx->phi_l[q], 0, n);
    if (!per) launch_boundary(ctx->st, gh, gl, n, 0, ctx->d_scal + 1, S, pair);
    launch_fill(ctx->st, gh, 0.0f, false);
    launch_fill(ctx->st, gl, 0.0f, false);
  }
  CKL();
  const bool m64 = ctx->cfg.precision == PM_MIXED_FP64;
  if (m64) m64_from_pairs(ctx, 0, n);  // zero interior, boundary values
  int guess = ctx->cfg.guess;
  ctx->cfg.guess = PM_GUESS_WARM;  // already zeroed
  st = solve(ctx);
  ctx->cfg.guess = guess;
  if (m64 && st == PM_OK) m64_to_pairs(ctx, 0, n);
  if (vcycles_out) *vcycles_out = ctx->vcycles_last;
  if (resid_out) *resid_out = ctx->resid_last;
  if (st != PM_OK) return st;
  double shift = 0.0;
  Grid ph = full_view(ctx, ctx->phi_h[ctx->cur], 0, n), pl = full_view(ctx, ctx->phi_l[ctx->cur], 0, n);
  if (per) {
    launch_sum_phi(ctx->st, ph, pl, ctx->partial, ctx->counter, ctx->d_scal + 12);
    CKL();
    st = sync_read(ctx);
    if (st != PM_OK) return st;
    shift = ctx->h_scal[12] / ((double)n * n * n);
  }
  launch_phi_out(ctx->st, ph, pl, phi_out_dev, phi64_out_dev, shift);
  CKL();
  CK(cudaStreamSynchronize(ctx->st));
  return PM_OK;
}

namespace {
pm_status deposit_any(bool tsc, const char* who, float* pos4_dev, const float* mom4_dev,
                      int64_t n, float drift_coef, int32_t n_mesh, int32_t lo, int32_t side,
                      int32_t periodic, int64_t* rho_dev, int64_t* escaped_out,
                      void* stream) {
  pm_ctx* ctx = nullptr;
  if ((!pos4_dev && n > 0) || !rho_dev || n < 0 || n_mesh < 1 || side < 1 || lo < 0 || lo + side > n_mesh)
    return fail(nullptr, PM_EINVAL, std::string(who) + ": bad argument");
  if (periodic && (lo != 0 || side != n_mesh))
    return fail(nullptr, PM_EINVAL, std::string(who) + ": periodic needs the whole mesh");
  cudaStream_t st = (cudaStream_t)stream;
  unsigned long long* esc = nullptr;
  CK(cudaMallocAsync((void**)&esc, sizeof(unsigned long long), st));
  CK(cudaMemsetAsync(esc, 0, sizeof(unsigned long long), st));
  if (tsc)
    launch_drift_deposit_tsc(st, n, (float4*)pos4_dev, (const float4*)mom4_dev, drift_coef,
                             mom4_dev != nullptr, n_mesh, lo, side, periodic,
                             (unsigned long long*)rho_dev, esc);
  else
    launch_drift_deposit(st, std::max(1, std::min(gkd_blocks(n) * 4, 152 * 16)),
                         (float4*)pos4_dev, (const float4*)mom4_dev, n, drift_coef,
                         mom4_dev != nullptr, n_mesh, lo, side, periodic,
                         (unsigned long long*)rho_dev, esc);
  CKL();
  if (escaped_out) {
    unsigned long long h = 0;
    CK(cudaMemcpyAsync(&h, esc, sizeof(h), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    *escaped_out = (int64_t)h;
  }
  CK(cudaFreeAsync(esc, st));
  return PM_OK;
}
}  // namespace

pm_status pm_deposit(float* pos4_dev, const float* mom4_dev, int64_t n, float drift_coef,
                     int32_t n_mesh, int32_t lo, int32_t side, int32_t periodic,
                     int64_t* rho_dev, int64_t* escaped_out, void* stream) {
  return deposit_any(false, "pm_deposit", pos4_dev, mom4_dev, n, drift_coef, n_mesh, lo, side,
                     periodic, rho_dev, escaped_out, stream);
}

pm_status pm_deposit_tsc(float* pos4_dev, const float* mom4_dev, int64_t n, float drift_coef,
                         int32_t n_mesh, int32_t lo, int32_t side, int32_t periodic,
                         int64_t* rho_dev, int64_t* escaped_out, void* stream) {
  return deposit_any(true, "pm_deposit_tsc", pos4_dev, mom4_dev, n, drift_coef, n_mesh, lo,
                     side, periodic, rho_dev, escaped_out, stream);
}

pm_status pm_sort_particles(const float* pos4_dev, const float* mom4_dev, int64_t n,
                            int32_t n_mesh, float* pos4_out, float* mom4_out, void* stream) {
  pm_ctx* ctx = nullptr;
  if (n < 0 || n >= (1LL << 31) || n_mesh < 1 || n_mesh > 1024)
    return fail(ctx, PM_EINVAL, "pm_sort_particles: n in [0, 2^31), n_mesh in [1, 1024]");
  if (n == 0) return PM_OK;
  if (!pos4_dev || !pos4_out || (mom4_dev && !mom4_out))
    return fail(ctx, PM_EINVAL, "pm_sort_particles: NULL argument");
  const size_t bytes = sizeof(float4) * (size_t)n;
  auto overlap = [&](const void* a, const void* b) {
    const char *x = (const char*)a, *y = (const char*)b;
    return a && b && x < y + bytes && y < x + bytes;
  };
  if (overlap(pos4_out, pos4_dev) || overlap(pos4_out, mom4_dev) ||
      (mom4_dev && (overlap(mom4_out, pos4_dev) || overlap(mom4_out, mom4_dev) ||
                    overlap(mom4_out, pos4_out))))
    return fail(ctx, PM_EINVAL, "pm_sort_particles: outputs overlap the inputs or each other");
  cudaStream_t st = (cudaStream_t)stream;
  SortWork w{};
  void** bufs[] = {(void**)&w.keys[0], (void**)&w.keys[1], (void**)&w.vals[0],
                   (void**)&w.vals[1], (void**)&w.counts, (void**)&w.ghist};
  const size_t sizes[] = {sizeof(unsigned) * (size_t)n, sizeof(unsigned) * (size_t)n,
                          sizeof(unsigned) * (size_t)n, sizeof(unsigned) * (size_t)n,
                          sizeof(unsigned) * sort_counts_len(n),
                          sizeof(unsigned) * sort_ghist_len()};
  auto release = [&]() {
    for (void** b : bufs)
      if (*b) cudaFree(*b);
  };
  for (int q = 0; q < 6; ++q) {
    if (cudaMalloc(bufs[q], sizes[q]) != cudaSuccess) {
      cudaGetLastError();
      release();
      return fail(ctx, PM_ENOMEM, "pm_sort_particles: cudaMalloc failed");
    }
  }
  cudaError_t e = launch_sort_particles(st, (const float4*)pos4_dev, (const float4*)mom4_dev, n,
                                        n_mesh, w, (float4*)pos4_out, (float4*)mom4_out);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  release();
  if (e != cudaSuccess)
    return fail(ctx, PM_ECUDA, std::string("pm_sort_particles: ") + cudaGetErrorString(e));
  return PM_OK;
}

namespace {
// Device work space of one P(k) call: CIC counts, contrast, its R2C
// transform, bin accumulators (3 per bin + the escape counter) and slopes.
struct PkWork {
  unsigned long long* rho = nullptr;
  float* delta = nullptr;
  cufftComplex* dk = nullptr;
  double* acc = nullptr;
  double* nu = nullptr;
  cufftHandle plan = 0;
  bool have_plan = false;
  ~PkWork() {
    if (have_plan) cufftDestroy(plan);
    cudaFree(rho);
    cudaFree(delta);
    cudaFree(dk);
    cudaFree(acc);
    cudaFree(nu);
  }
};

// CIC deposit of the particles on the periodic n_mesh^3 mesh, contrast,
// forward FFT into w.dk; w.acc cleared.
pm_status pk_transform(PkWork& w, const char* who, const float* pos4_dev, int64_t n,
                       int n_mesh, int n_bins, cudaStream_t st) {
  const size_t cells = (size_t)n_mesh * n_mesh * n_mesh;
  const size_t modes = (size_t)n_mesh * n_mesh * (n_mesh / 2 + 1);
  if (cudaMalloc((void**)&w.rho, sizeof(unsigned long long) * cells) != cudaSuccess ||
      cudaMalloc((void**)&w.delta, sizeof(float) * cells) != cudaSuccess ||
      cudaMalloc((void**)&w.dk, sizeof(cufftComplex) * modes) != cudaSuccess ||
      cudaMalloc((void**)&w.acc, sizeof(double) * (3 * n_bins + 1)) != cudaSuccess ||
      cudaMalloc((void**)&w.nu, sizeof(double) * n_bins) != cudaSuccess)
    return fail(nullptr, PM_ENOMEM, std::string(who) + ": cudaMalloc failed");
  cudaMemsetAsync(w.rho, 0, sizeof(unsigned long long) * cells, st);
  cudaMemsetAsync(w.acc, 0, sizeof(double) * (3 * n_bins + 1), st);
  // positions are read-only here: no drift
  launch_drift_deposit(st, std::max(1, std::min(gkd_blocks(n) * 4, 152 * 16)),
                       (float4*)pos4_dev, nullptr, n, 0.f, false, n_mesh, 0, n_mesh, 1, w.rho,
                       (unsigned long long*)(w.acc + 3 * n_bins));
  const double mean = (double)n * 281474976710656.0 / (double)cells;
  launch_pk_delta(st, w.rho, w.delta, n_mesh, 1.0 / mean);
  if (cufftPlan3d(&w.plan, n_mesh, n_mesh, n_mesh, CUFFT_R2C) != CUFFT_SUCCESS)
    return fail(nullptr, PM_ECUDA, std::string(who) + ": cufftPlan3d failed");
  w.have_plan = true;
  cufftSetStream(w.plan, st);
  if (cufftExecR2C(w.plan, w.delta, w.dk) != CUFFT_SUCCESS)
    return fail(nullptr, PM_ECUDA, std::string(who) + ": cufftExecR2C failed");
  return PM_OK;
}

// Binned (k, P, modes) from the accumulators (synchronises st), then clears them.
pm_status pk_read(PkWork& w, const char* who, int n_bins, cudaStream_t st, double* k_out,
                  double* pk_out, double* modes_out) {
  std::vector<double> h(3 * n_bins);
  if (cudaMemcpyAsync(h.data(), w.acc, sizeof(double) * 3 * n_bins, cudaMemcpyDeviceToHost,
                      st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return fail(nullptr, PM_ECUDA,
                std::string(who) + ": " + cudaGetErrorString(cudaGetLastError()));
  for (int b = 0; b < n_bins; ++b) {
    double c = h[3 * b];
    modes_out[b] = c;
    k_out[b] = c > 0 ? h[3 * b + 1] / c : NAN;
    pk_out[b] = c > 0 ? h[3 * b + 2] / c : NAN;
  }
  cudaMemsetAsync(w.acc, 0, sizeof(double) * 3 * n_bins, st);
  return PM_OK;
}

// Local slope d ln P / d ln k per bin: centred over bins b-1, b+1 (one-sided
// at the ends), the previous value kept where a P involved is not positive,
// clipped to [-6, 4].
void pk_slopes(const std::vector<double>& k, const std::vector<double>& p,
               std::vector<double>& nu) {
  const int nb = (int)p.size();
  std::vector<double> out = nu;
  for (int b = 0; b < nb; ++b) {
    const int lo = std::max(b - 1, 0), hi = std::min(b + 1, nb - 1);
    if (hi == lo) continue;
    if (p[lo] > 0 && p[hi] > 0 && k[lo] > 0 && k[hi] > 0)
      out[b] = std::log(p[hi] / p[lo]) / std::log(k[hi] / k[lo]);
  }
  for (int b = 0; b < nb; ++b) nu[b] = std::min(4.0, std::max(-6.0, out[b]));
}
}  // namespace

pm_status pm_power_spectrum(const float* pos4_dev, int64_t n, double box, int32_t n_mesh,
                            int32_t n_bins, int32_t subtract_shot, double* k_out,
                            double* pk_out, double* modes_out, void* stream) {
  if (!pos4_dev || n <= 0 || !(box > 0) || n_mesh < 2 || n_bins < 1 || n_bins > 2048 ||
      !k_out || !pk_out || !modes_out)
    return fail(nullptr, PM_EINVAL, "pm_power_spectrum: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  PkWork w;
  pm_status ret = pk_transform(w, "pm_power_spectrum", pos4_dev, n, n_mesh, n_bins, st);
  if (ret != PM_OK) return ret;
  const double shot = subtract_shot ? box * box * box / (double)n : 0.0;
  launch_pk_bin(st, (const float2*)w.dk, n_mesh, box, shot, n_bins, w.acc);
  return pk_read(w, "pm_power_spectrum", n_bins, st, k_out, pk_out, modes_out);
}

pm_status pm_power_spectrum_jing(const float* pos4_dev, int64_t n, double box, int32_t n_mesh,
                                 int32_t n_bins, int32_t subtract_shot, int32_t alias_range,
                                 int32_t max_iter, double tol, double* k_out, double* pk_out,
                                 double* modes_out, double* nu_out, int32_t* passes_out,
                                 void* stream) {
  if (!pos4_dev || n <= 0 || !(box > 0) || n_mesh < 2 || n_bins < 1 || n_bins > 2048 ||
      alias_range < 1 || alias_range > 3 || max_iter < 1 || !(tol > 0) || !k_out || !pk_out ||
      !modes_out)
    return fail(nullptr, PM_EINVAL, "pm_power_spectrum_jing: bad argument");
  const char* who = "pm_power_spectrum_jing";
  cudaStream_t st = (cudaStream_t)stream;
  PkWork w;
  pm_status ret = pk_transform(w, who, pos4_dev, n, n_mesh, n_bins, st);
  if (ret != PM_OK) return ret;
  const double shot = subtract_shot ? box * box * box / (double)n : 0.0;
  std::vector<double> k(n_bins), p(n_bins), c(n_bins), nu(n_bins, -1.0);
  // first-order estimate for the starting slopes
  launch_pk_bin(st, (const float2*)w.dk, n_mesh, box, shot, n_bins, w.acc);
  ret = pk_read(w, who, n_bins, st, k.data(), p.data(), c.data());
  if (ret != PM_OK) return ret;
  pk_slopes(k, p, nu);
  int passes = 0;
  for (passes = 1; passes <= max_iter; ++passes) {
    if (cudaMemcpyAsync(w.nu, nu.data(), sizeof(double) * n_bins, cudaMemcpyHostToDevice,
                        st) != cudaSuccess)
      return fail(nullptr, PM_ECUDA, std::string(who) + ": uploading slopes failed");
    launch_pk_jing(st, (const float2*)w.dk, n_mesh, box, shot, n_bins, alias_range, w.nu,
                   w.acc);
    ret = pk_read(w, who, n_bins, st, k.data(), p.data(), c.data());
    if (ret != PM_OK) return ret;
    std::vector<double> nn = nu;
    pk_slopes(k, p, nn);
    double dmax = 0.0;
    for (int b = 0; b < n_bins; ++b) dmax = std::max(dmax, std::fabs(nn[b] - nu[b]));
    nu = nn;
    if (dmax < tol) break;
  }
  for (int b = 0; b < n_bins; ++b) {
    k_out[b] = k[b];
    pk_out[b] = p[b];
    modes_out[b] = c[b];
    if (nu_out) nu_out[b] = nu[b];
  }
  if (passes_out) *passes_out = std::min(passes, (int)max_iter);
  return PM_OK;
}

pm_status pm_stats(pm_ctx* ctx, pm_stats_t* o) {
  if (!ctx || !o) return fail(ctx, PM_EINVAL, "pm_stats: NULL argument");
  pm_status st = sync_read(ctx);
  if (st != PM_OK) return st;
  o->step = ctx->step;
  o->a = ctx->a[ctx->step];
  o->n_active = ctx->n_active;
  o->n_lightcone = ctx->n_lc;
  o->cube_lo = ctx->lo;
  o->cube_side = ctx->s;
  o->periodic = ctx->periodic;
  o->vcycles_last = ctx->vcycles_last;
  o->vcycles_total = ctx->vcycles_total;
  o->resid_last = ctx->resid_last;
  o->escaped = (int64_t)ctx->h_cnt[1];
  o->particle_steps = ctx->particle_steps;
  o->guess_used_last = ctx->guess_used_last;
  o->guess_used_total = ctx->guess_used_total;
  o->resid_start = ctx->resid_start;
  o->resid_guess = ctx->resid_guess;
  return PM_OK;
}

pm_status pm_set_guess(pm_ctx* ctx, pm_guess* net) {
  if (!ctx) return fail(nullptr, PM_EINVAL, "pm_set_guess: NULL context");
  if (net && !ctx->nn_in) {
    const size_t bytes = sizeof(float) * (size_t)ctx->n * ctx->n * ctx->n;
    pm_status st = alloc(ctx, (void**)&ctx->nn_in, bytes);
    if (st == PM_OK) st = alloc(ctx, (void**)&ctx->nn_out, bytes);
    if (st != PM_OK) return st;
  }
  CK(cudaDeviceSynchronize());  // parameters written on the network's stream
  ctx->net = net;
  return PM_OK;
}

pm_status pm_capture(pm_ctx* ctx, float* r_dev, float* e_dev) {
  if (!ctx) return fail(nullptr, PM_EINVAL, "pm_capture: NULL context");
  if ((r_dev == nullptr) != (e_dev == nullptr))
    return fail(ctx, PM_EINVAL, "pm_capture: give both arrays or neither");
  if (r_dev && ctx->cfg.precision != PM_MIXED)
    return fail(ctx, PM_EINVAL, "pm_capture: needs PM_MIXED");
  ctx->cap_r = r_dev;
  ctx->cap_e = e_dev;
  return PM_OK;
}

pm_status pm_schedule(pm_ctx* ctx, double* a, double* dtau, double* a_half, double* chi) {
  if (!ctx) return fail(nullptr, PM_EINVAL, "pm_schedule: NULL context");
  size_t m = ctx->a.size();
  if (a) std::copy(ctx->a.begin(), ctx->a.end(), a);
  if (dtau) std::copy(ctx->dtau.begin(), ctx->dtau.begin() + m, dtau);
  if (a_half) std::copy(ctx->a_half.begin(), ctx->a_half.begin() + m, a_half);
  if (chi) std::copy(ctx->chi.begin(), ctx->chi.end(), chi);
  return PM_OK;
}

pm_status pm_get_particles(pm_ctx* ctx, float* pos4, float* mom4, int32_t host_mem,
                           int64_t* n_active_out) {
  if (!ctx) return fail(nullptr, PM_EINVAL, "pm_get_particles: NULL context");
  cudaMemcpyKind kind = host_mem ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  size_t bytes = sizeof(float4) * ctx->n_active;
  if (pos4 && bytes) CK(cudaMemcpyAsync(pos4, ctx->pos, bytes, kind, ctx->st));
  if (mom4 && bytes) CK(cudaMemcpyAsync(mom4, ctx->mom, bytes, kind, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  if (n_active_out) *n_active_out = ctx->n_active;
  return PM_OK;
}

pm_status pm_set_particles(pm_ctx* ctx, const float* pos4, const float* mom4, int64_t n,
                           int32_t host_mem) {
  if (!ctx) return fail(nullptr, PM_EINVAL, "pm_set_particles: NULL context");
  if (!pos4 || !mom4 || n < 0 || n > ctx->N0)
    return fail(ctx, PM_EINVAL, "pm_set_particles: bad argument");
  cudaMemcpyKind kind = host_mem ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  size_t bytes = sizeof(float4) * n;
  if (bytes) {
    CK(cudaMemcpyAsync(ctx->pos, pos4, bytes, kind, ctx->st));
    CK(cudaMemcpyAsync(ctx->mom, mom4, bytes, kind, ctx->st));
  }
  ctx->n_active = n;
  return PM_OK;
}

pm_status pm_get_lightcone(pm_ctx* ctx, float* pos4, float* mom4, int32_t host_mem,
                           int64_t* n_out) {
  if (!ctx) return fail(nullptr, PM_EINVAL, "pm_get_lightcone: NULL context");
  cudaMemcpyKind kind = host_mem ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  size_t bytes = sizeof(float4) * ctx->n_lc;
  if (pos4 && bytes) CK(cudaMemcpyAsync(pos4, ctx->lc_pos, bytes, kind, ctx->st));
  if (mom4 && bytes) CK(cudaMemcpyAsync(mom4, ctx->lc_mom, bytes, kind, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  if (n_out) *n_out = ctx->n_lc;
  return PM_OK;
}

pm_status pm_get_forces(pm_ctx* ctx, float* f4, int32_t host_mem, int64_t* n_out) {
  if (!ctx) return fail(nullptr, PM_EINVAL, "pm_get_forces: NULL context");
  if (!ctx->forces || !ctx->forces_valid)
    return fail(ctx, PM_EINVAL, "pm_get_forces: store_forces is off or no step ran");
  cudaMemcpyKind kind = host_mem ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (f4 && ctx->forces_n)
    CK(cudaMemcpyAsync(f4, ctx->forces, sizeof(float4) * ctx->forces_n, kind, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  if (n_out) *n_out = ctx->forces_n;
  return PM_OK;
}

namespace {
// Checkpoint layout: this header, then pos and mom of the active particles,
// the lightcone pos and mom, then phi_hi, phi_lo (the current buffer),
// prev_hi, prev_lo (full (n+2)^3 arrays).
struct CkptHeader {
  char magic[8];
  uint32_t version, header_bytes;
  pm_config cfg;
  int32_t step, cur, n_sol, field_ready, vc_prev, cube_valid, lo, s, periodic, vcycles_last;
  int64_t n_active, n_lc, vcycles_total, particle_steps, escaped, guess_used_total;
  double ah_hist[2], resid_last, resid_start, resid_guess;
  uint64_t padded;
};
const char CKPT_MAGIC[8] = {'P', 'M', 'S', 'H', 'R', 'K', 'C', '1'};

bool cfg_equal(const pm_config& a, const pm_config& b) {
  return a.n_mesh == b.n_mesh && a.n_particles == b.n_particles && a.box_mpch == b.box_mpch &&
         a.omega_m == b.omega_m && a.omega_l == b.omega_l && a.a_init == b.a_init &&
         a.a_final == b.a_final && a.n_steps == b.n_steps && a.rtol == b.rtol &&
         a.max_vcycles == b.max_vcycles && a.precision == b.precision && a.guess == b.guess &&
         a.bc == b.bc && a.shrink == b.shrink && a.buffer_cells == b.buffer_cells &&
         a.store_forces == b.store_forces && a.gravity == b.gravity &&
         a.c_eff_factor == b.c_eff_factor && a.assignment == b.assignment &&
         a.domain == b.domain && a.sort_every == b.sort_every &&
         a.inner_vcycles == b.inner_vcycles;
}

// device <-> file through a bounded host buffer
constexpr size_t CKPT_CHUNK = size_t(64) << 20;
bool dev_to_file(FILE* f, const void* dev, size_t bytes, std::vector<char>& buf) {
  for (size_t off = 0; off < bytes; off += CKPT_CHUNK) {
    const size_t m = std::min(CKPT_CHUNK, bytes - off);
    if (cudaMemcpy(buf.data(), (const char*)dev + off, m, cudaMemcpyDeviceToHost) != cudaSuccess)
      return false;
    if (std::fwrite(buf.data(), 1, m, f) != m) return false;
  }
  return true;
}
bool file_to_dev(FILE* f, void* dev, size_t bytes, std::vector<char>& buf) {
  for (size_t off = 0; off < bytes; off += CKPT_CHUNK) {
    const size_t m = std::min(CKPT_CHUNK, bytes - off);
    if (std::fread(buf.data(), 1, m, f) != m) return false;
    if (cudaMemcpy((char*)dev + off, buf.data(), m, cudaMemcpyHostToDevice) != cudaSuccess)
      return false;
  }
  return true;
}
}  // namespace

pm_status pm_get_potential(pm_ctx* ctx, double* phi_host, int32_t* lo_out, int32_t* side_out) {
  if (!ctx) return fail(nullptr, PM_EINVAL, "pm_get_potential: NULL context");
  const int P = ctx->P, lo = ctx->lo, s = ctx->s;
  const size_t padded = (size_t)P * P * P;
  const bool m64 = ctx->cfg.precision == PM_MIXED_FP64;
  std::vector<float> hi(m64 ? 0 : padded), lo_(m64 ? 0 : padded);
  std::vector<double> d64(m64 ? padded : 0);
  if (m64) {
    CK(cudaMemcpyAsync(d64.data(), ctx->phi64, sizeof(double) * padded, cudaMemcpyDeviceToHost,
                       ctx->st));
  } else {
    CK(cudaMemcpyAsync(hi.data(), ctx->phi_h[ctx->cur], sizeof(float) * padded,
                       cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaMemcpyAsync(lo_.data(), ctx->phi_l[ctx->cur], sizeof(float) * padded,
                       cudaMemcpyDeviceToHost, ctx->st));
  }
  CK(cudaStreamSynchronize(ctx->st));
  if (phi_host) {
    const int Q = s + 2;
    for (int k = 0; k < Q; ++k)
      for (int j = 0; j < Q; ++j)
        for (int i = 0; i < Q; ++i) {
          size_t src = ((size_t)(lo + k) * P + (lo + j)) * P + (lo + i);
          phi_host[((size_t)k * Q + j) * Q + i] =
              m64 ? d64[src] : (double)hi[src] + (double)lo_[src];
        }
  }
  if (lo_out) *lo_out = lo;
  if (side_out) *side_out = s;
  return PM_OK;
}

pm_status pm_save(pm_ctx* ctx, const char* path) {
  if (!ctx || !path) return fail(ctx, PM_EINVAL, "pm_save: NULL argument");
  pm_status st = sync_read(ctx);  // completes the stream; escaped count
  if (st != PM_OK) return st;
  CkptHeader h;
  std::memset(&h, 0, sizeof h);
  std::memcpy(h.magic, CKPT_MAGIC, 8);
  h.version = 1;
  h.header_bytes = (uint32_t)sizeof h;
  h.cfg = ctx->cfg;
  h.step = ctx->step;
  h.cur = ctx->cur;
  h.n_sol = ctx->n_sol;
  h.field_ready = ctx->field_ready ? 1 : 0;
  h.vc_prev = ctx->vc_prev;
  h.cube_valid = ctx->cube_valid ? 1 : 0;
  h.lo = ctx->lo;
  h.s = ctx->s;
  h.periodic = ctx->periodic;
  h.vcycles_last = ctx->vcycles_last;
  h.n_active = ctx->n_active;
  h.n_lc = ctx->n_lc;
  h.vcycles_total = ctx->vcycles_total;
  h.particle_steps = ctx->particle_steps;
  h.escaped = (int64_t)ctx->h_cnt[1];
  h.guess_used_total = ctx->guess_used_total;
  h.ah_hist[0] = ctx->ah_hist[0];
  h.ah_hist[1] = ctx->ah_hist[1];
  h.resid_last = ctx->resid_last;
  h.resid_start = ctx->resid_start;
  h.resid_guess = ctx->resid_guess;
  h.padded = (uint64_t)ctx->P * ctx->P * ctx->P;
  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(ctx, PM_EIO, std::string("pm_save: cannot open ") + path);
  std::vector<char> buf(CKPT_CHUNK);
  const size_t pb = sizeof(float4), gb = sizeof(float) * (size_t)h.padded;
  // PM_MIXED_FP64 keeps its potential in FP64: those two arrays instead of
  // the four pair arrays (the same byte count)
  const bool m64 = ctx->cfg.precision == PM_MIXED_FP64;
  bool ok = std::fwrite(&h, sizeof h, 1, f) == 1 &&
            dev_to_file(f, ctx->pos, pb * h.n_active, buf) &&
            dev_to_file(f, ctx->mom, pb * h.n_active, buf) &&
            dev_to_file(f, ctx->lc_pos, pb * h.n_lc, buf) &&
            dev_to_file(f, ctx->lc_mom, pb * h.n_lc, buf) &&
            (m64 ? dev_to_file(f, ctx->phi64, 2 * gb, buf) &&
                       dev_to_file(f, ctx->prev64, 2 * gb, buf)
                 : dev_to_file(f, ctx->phi_h[ctx->cur], gb, buf) &&
                       dev_to_file(f, ctx->phi_l[ctx->cur], gb, buf) &&
                       dev_to_file(f, ctx->prev_hi, gb, buf) &&
                       dev_to_file(f, ctx->prev_lo, gb, buf));
  ok = (std::fclose(f) == 0) && ok;
  if (!ok) return fail(ctx, PM_EIO, std::string("pm_save: writing ") + path + " failed");
  return PM_OK;
}

pm_status pm_load(pm_ctx* ctx, const char* path) {
  if (!ctx || !path) return fail(ctx, PM_EINVAL, "pm_load: NULL argument");
  CK(cudaStreamSynchronize(ctx->st));
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(ctx, PM_EIO, std::string("pm_load: cannot open ") + path);
  CkptHeader h;
  if (std::fread(&h, sizeof h, 1, f) != 1) {
    std::fclose(f);
    return fail(ctx, PM_EIO, "pm_load: short header");
  }
  const uint64_t padded = (uint64_t)ctx->P * ctx->P * ctx->P;
  if (std::memcmp(h.magic, CKPT_MAGIC, 8) != 0 || h.version != 1 ||
      h.header_bytes != sizeof h || h.padded != padded) {
    std::fclose(f);
    return fail(ctx, PM_EINVAL, "pm_load: not a checkpoint of this library and mesh");
  }
  if (!cfg_equal(h.cfg, ctx->cfg)) {
    std::fclose(f);
    return fail(ctx, PM_EINVAL, "pm_load: the checkpoint has another configuration");
  }
  if (h.step < 0 || h.step > ctx->cfg.n_steps || h.n_active < 0 || h.n_lc < 0 ||
      h.n_active > ctx->N0 || h.n_lc > ctx->N0 ||  // the record mode keeps both
      (ctx->cfg.shrink != PM_SHRINK_RECORD && h.n_active + h.n_lc > ctx->N0) ||
      (h.cur != 0 && h.cur != 1) || h.n_sol < 0 || h.vc_prev < 0 ||
      h.vc_prev > ctx->cfg.max_vcycles || h.vcycles_last < 0 ||
      (h.field_ready != 0 && h.field_ready != 1) || (h.cube_valid != 0 && h.cube_valid != 1)) {
    std::fclose(f);
    return fail(ctx, PM_EINVAL, "pm_load: inconsistent checkpoint header");
  }
  if (h.cube_valid) {
    // the active cube is a function of the schedule: the one of the last
    // completed step (or of the step that stopped early); anything else
    // would index the level arrays outside their allocations
    bool match = false;
    for (int k = std::max(0, h.step - 1); k <= h.step && k <= ctx->cfg.n_steps; ++k) {
      int lo, s, per;
      geometry(ctx, ctx->R[k], &lo, &s, &per);
      match = match || (lo == h.lo && s == h.s && per == h.periodic);
    }
    if (!match) {
      std::fclose(f);
      return fail(ctx, PM_EINVAL, "pm_load: the checkpoint's active cube does not belong to "
                                  "its step");
    }
  }
  std::vector<char> buf(CKPT_CHUNK);
  const size_t pb = sizeof(float4), gb = sizeof(float) * (size_t)padded;
  const bool m64 = ctx->cfg.precision == PM_MIXED_FP64;
  bool ok = file_to_dev(f, ctx->pos, pb * h.n_active, buf) &&
            file_to_dev(f, ctx->mom, pb * h.n_active, buf) &&
            file_to_dev(f, ctx->lc_pos, pb * h.n_lc, buf) &&
            file_to_dev(f, ctx->lc_mom, pb * h.n_lc, buf) &&
            (m64 ? file_to_dev(f, ctx->phi64, 2 * gb, buf) &&
                       file_to_dev(f, ctx->prev64, 2 * gb, buf)
                 : file_to_dev(f, ctx->phi_h[h.cur], gb, buf) &&
                       file_to_dev(f, ctx->phi_l[h.cur], gb, buf) &&
                       file_to_dev(f, ctx->prev_hi, gb, buf) &&
                       file_to_dev(f, ctx->prev_lo, gb, buf));
  std::fclose(f);
  if (!ok) return fail(ctx, PM_EIO, std::string("pm_load: reading ") + path + " failed");
  ctx->step = h.step;
  ctx->cur = h.cur;
  ctx->n_sol = h.n_sol;
  ctx->field_ready = h.field_ready != 0;
  ctx->vc_prev = h.vc_prev;
  ctx->vcycles_last = h.vcycles_last;
  ctx->n_active = h.n_active;
  ctx->n_lc = h.n_lc;
  ctx->vcycles_total = h.vcycles_total;
  ctx->particle_steps = h.particle_steps;
  ctx->guess_used_total = h.guess_used_total;
  ctx->ah_hist[0] = h.ah_hist[0];
  ctx->ah_hist[1] = h.ah_hist[1];
  ctx->resid_last = h.resid_last;
  ctx->resid_start = h.resid_start;
  ctx->resid_guess = h.resid_guess;
  ctx->forces_valid = false;
  drop_graph(ctx);
  unsigned long long cnt[4] = {0ull, (unsigned long long)h.escaped, 0ull, 0ull};
  CK(cudaMemcpy(ctx->d_cnt, cnt, sizeof cnt, cudaMemcpyHostToDevice));
  ctx->cube_valid = false;
  if (h.cube_valid) {
    // the cube of the last step, its levels and mean-density term, so that
    // the next step sees no change of boundary phase
    pm_status st = set_cube(ctx, h.lo, h.s, h.periodic, ctx->R[ctx->step]);
    if (st != PM_OK) return st;
  }
  CK(cudaStreamSynchronize(ctx->st));
  return sync_read(ctx);
}

pm_status pm_profile(pm_ctx* ctx, int32_t enable) {
  if (!ctx) return fail(nullptr, PM_EINVAL, "pm_profile: NULL context");
  CK(cudaStreamSynchronize(ctx->st));
  prof_flush(ctx);
  if (enable && ctx->ev.empty()) {
    ctx->ev.resize(2 * EV_POOL);
    for (auto& e : ctx->ev) CK(cudaEventCreate(&e));
  }
  for (int c = 0; c < PM_PROF_N; ++c) {
    ctx->prof_ms[c] = 0.0;
    ctx->prof_groups[c] = 0;
    ctx->prof_bytes[c] = 0.0;
  }
  ctx->prof_on = enable != 0;
  return PM_OK;
}

pm_status pm_profile_read(pm_ctx* ctx, int32_t cls, double* ms, int64_t* groups,
                          double* bytes) {
  if (!ctx || cls < 0 || cls >= PM_PROF_N) return fail(ctx, PM_EINVAL, "pm_profile_read");
  CK(cudaStreamSynchronize(ctx->st));
  prof_flush(ctx);
  if (ms) *ms = ctx->prof_ms[cls];
  if (groups) *groups = ctx->prof_groups[cls];
  if (bytes) *bytes = ctx->prof_bytes[cls];
  return PM_OK;
}

int64_t pm_launch_count(void) { return g_launches.load(); }

pm_status pm_smoother_tiles(pm_ctx* ctx, int32_t* sides, int32_t* tile_height,
                            int32_t* z_chunk, int32_t cap, int32_t* count) {
  if (!ctx || !count || cap < 0) return fail(ctx, PM_EINVAL, "pm_smoother_tiles: bad argument");
  const int m = (int)ctx->f2_pick.size();
  for (int i = 0; i < m && i < cap; ++i) {
    if (sides) sides[i] = ctx->f2_pick[i].s;
    if (tile_height) tile_height[i] = ctx->f2_pick[i].ty;
    if (z_chunk) z_chunk[i] = ctx->f2_pick[i].zc;
  }
  *count = m;
  return PM_OK;
}

int32_t pm_mg_cluster_size(void) { return cmg_cluster(); }

const char* pm_last_error(const pm_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_err.c_str();
}

void pm_destroy(pm_ctx* ctx) {
  if (!ctx) return;
  if (ctx->st) cudaStreamSynchronize(ctx->st);
  void* ptrs[] = {ctx->pos, ctx->mom, ctx->pos2, ctx->mom2, ctx->lc_pos, ctx->lc_mom,
                  ctx->forces, ctx->flags, ctx->block_keep, ctx->keep_off, ctx->rho,
                  ctx->phi_h[0], ctx->phi_l[0], ctx->phi_h[1], ctx->phi_l[1], ctx->f_hi,
                  ctx->f_lo, ctx->prev_hi, ctx->prev_lo,
                  ctx->partial, ctx->partial_m,
                  ctx->counter, ctx->d_scal, ctx->bgm, ctx->d_cnt, ctx->ballw,
                  ctx->nn_in, ctx->nn_out, ctx->grad, ctx->sortw.keys[0], ctx->sortw.keys[1],
                  ctx->sortw.vals[0], ctx->sortw.vals[1], ctx->sortw.counts, ctx->sortw.ghist};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (float* p : ctx->lu) if (p) cudaFree(p);
  for (float* p : ctx->lb) if (p) cudaFree(p);
  for (float* p : ctx->lu2) if (p) cudaFree(p);
  for (double* p : ctx->lu64) if (p) cudaFree(p);
  for (double* p : ctx->lb64) if (p) cudaFree(p);
  if (ctx->phi64) cudaFree(ctx->phi64);
  if (ctx->prev64) cudaFree(ctx->prev64);
  if (ctx->ecorr) cudaFree(ctx->ecorr);
  if (ctx->f64) cudaFree(ctx->f64);
  drop_graph(ctx);
  for (auto& e : ctx->ev) cudaEventDestroy(e);
  if (ctx->h_scal) cudaFreeHost(ctx->h_scal);
  if (ctx->h_cnt) cudaFreeHost(ctx->h_cnt);
  delete ctx;
}

}  // extern "C"

// ===========================================================================
// Batched step: R realisations, one launch per phase, one V-cycle graph.
// ===========================================================================
namespace {

// Device-resident descriptor table of one batched launch, with a pinned
// staging copy on the host.
struct BTab {
  void* d_desc = nullptr;
  BTable* d_tab = nullptr;
  void* h_desc = nullptr;
  BTable* h_tab = nullptr;
  size_t desc_size = 0;
  int grid_max = 0;  // largest block total seen (graph launches use it)
};

}  // namespace

struct pm_batch {
  int R = 0;
  cudaStream_t st = nullptr;
  std::vector<pm_ctx*> ctx;
  int* d_active = nullptr;  // the graph solve's per-realisation activity
  double* d_scal = nullptr;  // 16 per realisation: [0] ||f||^2, [1..10] moments, [11] ||r||^2
  double* h_scal = nullptr;
  unsigned long long* d_cnt = nullptr;  // 4 per realisation: [0] survivors
  unsigned long long* h_cnt = nullptr;
  int* d_ovf = nullptr;
  BTab t_dep, t_src, t_bnd, t_pred, t_def, t_grad, t_gat, t_scan, t_scat;
  std::vector<BTab> t_vc;  // V-cycle launch slots
  int maxLc = 0;
  bool tables_stale = true;
  // the graph solve: init, defect, decision, a conditional while loop over
  // (V-cycle, defect, decision), the gradient field; one launch per solve
  cudaGraphExec_t sgraph = nullptr;
  cudaStream_t st2 = nullptr;  // captures the loop's body
  long long loop_kernels = 0;  // kernels of one pass of the loop body
  int rb_bx = 32, rb_by = 8;  // block shape of the batched colour pass (autotuned)
  bool rb_tuned = false;
  // the persistent solve: one cooperative launch per solve
  bool persistent = false;
  double wait_s = 2.0;         // longest wait at one grid barrier
  int extra = 0;               // barrier arrivals that never come (tests the wait limit)
  GridBar* d_bar = nullptr;
  GridBar* h_bar = nullptr;
  int* d_iters = nullptr;      // [0, MAX_REAL): V-cycles, [MAX_REAL, 2 MAX_REAL): failed
  int* h_iters = nullptr;
  double* d_rel = nullptr;     // [0, MAX_REAL): last relative residual, then rtol
  double* h_rel = nullptr;
  int* d_maxv = nullptr;
  SolveSlot* d_slots = nullptr;
  int n_slots_dev = 0;
  bool solved_on_device = false;  // this step's solve awaits its read-back
  std::string err;
};

namespace {

pm_status bfail(pm_batch* b, pm_status code, const std::string& msg) {
  if (b) b->err = msg; else g_err = msg;
  return code;
}

pm_status tab_alloc(pm_batch* B, BTab& t, size_t desc_size) {
  t.desc_size = desc_size;
  if (cudaMalloc(&t.d_desc, desc_size * MAX_MEMBERS) != cudaSuccess ||
      cudaMalloc((void**)&t.d_tab, sizeof(BTable)) != cudaSuccess ||
      cudaMallocHost(&t.h_desc, desc_size * MAX_MEMBERS) != cudaSuccess ||
      cudaMallocHost((void**)&t.h_tab, sizeof(BTable)) != cudaSuccess)
    return bfail(B, PM_ENOMEM, "pm_batch: table allocation failed");
  t.h_tab->m = 0;
  t.h_tab->off[0] = 0;
  return PM_OK;
}

void tab_free(BTab& t) {
  if (t.d_desc) cudaFree(t.d_desc);
  if (t.d_tab) cudaFree(t.d_tab);
  if (t.h_desc) cudaFreeHost(t.h_desc);
  if (t.h_tab) cudaFreeHost(t.h_tab);
  t = BTab();
}

// Stage descriptors (with their block counts) and upload; returns the block
// total.  The staging buffers are reused only after the stream has passed
// the previous upload (every batched phase is followed by a sync before the
// same table is rebuilt).
template <class D>
int tab_upload(pm_batch* B, BTab& t, const std::vector<D>& d, const std::vector<int>& blocks) {
  const int m = std::min((int)d.size(), MAX_MEMBERS);  // callers add <= 2 per realisation
  std::memcpy(t.h_desc, d.data(), sizeof(D) * m);
  t.h_tab->m = m;
  t.h_tab->off[0] = 0;
  for (int q = 0; q < m; ++q) t.h_tab->off[q + 1] = t.h_tab->off[q] + blocks[q];
  if (m) cudaMemcpyAsync(t.d_desc, t.h_desc, sizeof(D) * m, cudaMemcpyHostToDevice, B->st);
  cudaMemcpyAsync(t.d_tab, t.h_tab, sizeof(BTable), cudaMemcpyHostToDevice, B->st);
  int tot = t.h_tab->off[m];
  if (tot > t.grid_max) t.grid_max = tot;
  return tot;
}

int nblocks(dim3 g) { return (int)(g.x * g.y * g.z); }

template <class D>
void set_dims(D& d, int r, dim3 g) {
  d.r = r;
  d.gx = (int)g.x;
  d.gy = (int)g.y;
  d.gz = (int)g.z;
}

int first_small_level(const pm_ctx* c) {
  int L = (int)c->ls.size() - 1, Lc = 0;
  while (Lc < L && c->ls[Lc] > cmg_top_side(cmg_cluster())) ++Lc;
  return Lc;
}

float level_gam(int l) {
  float H = (float)(1 << l);
  return (H - 1.0f) / (H + 1.0f);
}

// V-cycle slot layout: down (4 sweeps + restriction per level), bottom, up
// (prolongation + 4 sweeps per level).
int slot_down(int l, int k) { return 5 * l + k; }            // k: 0..3 sweeps, 4 restrict
int slot_bottom(int maxLc) { return 5 * maxLc; }
int slot_up(int maxLc, int l, int k) { return 5 * maxLc + 1 + 5 * l + k; }  // k: 0 prolong, 1..4 sweeps
int n_slots(int maxLc) { return 10 * maxLc + 1; }

// Upload the descriptor tables of every V-cycle slot for the current cubes.
void upload_vcycle_tables(pm_batch* B) {
  const int R = B->R, M = B->maxLc;
  for (int l = 0; l < M; ++l) {
    for (int k = 0; k < 5; ++k) {  // down
      std::vector<int> bl;
      if (k < 4) {
        std::vector<RbgsDesc> d;
        for (int r = 0; r < R; ++r) {
          pm_ctx* c = B->ctx[r];
          if (l >= first_small_level(c)) continue;
          RbgsDesc e{};
          e.u = compact_view(c->lu[l], c->ls[l]);
          e.b = compact_view(c->lb[l], c->ls[l]);
          e.h2 = (float)(1 << (2 * l));
          e.gam = level_gam(l);
          e.color = k & 1;
          e.periodic = c->periodic;
          // level 0: e is not cleared (the first red sweep takes it as zero,
          // the black one after it its own cells); coarser: the restriction
          // zeroed it
          e.zero_start = k == 0 ? 1 : (k == 1 ? 2 : 0);
          set_dims(e, r, rbgs_grid_b(c->ls[l], B->rb_bx, B->rb_by));
          d.push_back(e);
          bl.push_back(nblocks(rbgs_grid_b(c->ls[l], B->rb_bx, B->rb_by)));
        }
        tab_upload(B, B->t_vc[slot_down(l, k)], d, bl);
      } else {
        std::vector<RestrictDesc> d;
        for (int r = 0; r < R; ++r) {
          pm_ctx* c = B->ctx[r];
          if (l >= first_small_level(c)) continue;
          RestrictDesc e{};
          e.u = compact_view(c->lu[l], c->ls[l]);
          e.b = compact_view(c->lb[l], c->ls[l]);
          e.uc = compact_view(c->lu[l + 1], c->ls[l + 1]);
          e.bc = compact_view(c->lb[l + 1], c->ls[l + 1]);
          e.inv_h2 = 1.0f / (float)(1 << (2 * l));
          e.gam = level_gam(l);
          e.periodic = c->periodic;
          set_dims(e, r, full_grid_b(c->ls[l + 1]));
          d.push_back(e);
          bl.push_back(nblocks(full_grid_b(c->ls[l + 1])));
        }
        tab_upload(B, B->t_vc[slot_down(l, k)], d, bl);
      }
    }
  }
  {  // bottom
    std::vector<CmgDesc> d;
    std::vector<int> bl;
    for (int r = 0; r < R; ++r) {
      pm_ctx* c = B->ctx[r];
      int Lc = first_small_level(c);
      CmgDesc e{};
      e.u = compact_view(c->lu[Lc], c->ls[Lc]);
      e.b = compact_view(c->lb[Lc], c->ls[Lc]);
      e.level = Lc;
      e.periodic = c->periodic;
      e.sweeps = COARSE_SWEEPS;
      e.zero_top = 1;
      set_dims(e, r, dim3(1, 1, 1));
      d.push_back(e);
      bl.push_back(1);
    }
    tab_upload(B, B->t_vc[slot_bottom(M)], d, bl);
  }
  for (int l = 0; l < M; ++l) {
    for (int k = 0; k < 5; ++k) {  // up
      std::vector<int> bl;
      if (k == 0) {
        std::vector<ProlongDesc> d;
        for (int r = 0; r < R; ++r) {
          pm_ctx* c = B->ctx[r];
          if (l >= first_small_level(c)) continue;
          ProlongDesc e{};
          e.uc = compact_view(c->lu[l + 1], c->ls[l + 1]);
          e.u = compact_view(c->lu[l], c->ls[l]);
          e.gam_c = level_gam(l + 1);
          e.periodic = c->periodic;
          set_dims(e, r, full_grid_b(c->ls[l]));
          d.push_back(e);
          bl.push_back(nblocks(full_grid_b(c->ls[l])));
        }
        tab_upload(B, B->t_vc[slot_up(M, l, k)], d, bl);
      } else {
        std::vector<RbgsDesc> d;
        for (int r = 0; r < R; ++r) {
          pm_ctx* c = B->ctx[r];
          if (l >= first_small_level(c)) continue;
          RbgsDesc e{};
          e.u = compact_view(c->lu[l], c->ls[l]);
          e.b = compact_view(c->lb[l], c->ls[l]);
          e.h2 = (float)(1 << (2 * l));
          e.gam = level_gam(l);
          e.color = (k - 1) & 1;
          e.periodic = c->periodic;
          e.zero_start = 0;
          set_dims(e, r, rbgs_grid_b(c->ls[l], B->rb_bx, B->rb_by));
          d.push_back(e);
          bl.push_back(nblocks(rbgs_grid_b(c->ls[l], B->rb_bx, B->rb_by)));
        }
        tab_upload(B, B->t_vc[slot_up(M, l, k)], d, bl);
      }
    }
  }
}

// Launch the V-cycle slots (captured once into a graph, grids at their
// largest; members and their grids come from the tables).
void launch_vcycle_slots(pm_batch* B, cudaStream_t st) {
  const int M = B->maxLc;
  const int* act = B->d_active;
  for (int l = 0; l < M; ++l) {
    for (int k = 0; k < 4; ++k) {
      BTab& t = B->t_vc[slot_down(l, k)];
      launch_rbgs_b(st, t.grid_max, (const RbgsDesc*)t.d_desc, t.d_tab, act, B->rb_bx,
                    B->rb_by);
    }
    BTab& t = B->t_vc[slot_down(l, 4)];
    launch_restrict_b(st, t.grid_max, (const RestrictDesc*)t.d_desc, t.d_tab, act);
  }
  BTab& tb = B->t_vc[slot_bottom(M)];
  // one cluster per realisation, shared memory for the largest top level
  launch_cmg_b(st, B->R, cmg_top_side(cmg_cluster()), (const CmgDesc*)tb.d_desc, act);
  for (int l = M - 1; l >= 0; --l) {
    BTab& tp = B->t_vc[slot_up(M, l, 0)];
    launch_prolong_b(st, tp.grid_max, (const ProlongDesc*)tp.d_desc, tp.d_tab, act);
    for (int k = 1; k < 5; ++k) {
      BTab& t = B->t_vc[slot_up(M, l, k)];
      launch_rbgs_b(st, t.grid_max, (const RbgsDesc*)t.d_desc, t.d_tab, act, B->rb_bx,
                    B->rb_by);
    }
  }
}

// Autotuner of the batched colour pass: before the V-cycle graph is
// captured, the down-sweep passes of every level run with each candidate
// block shape on the batch's own grids (they only write the levels'
// iterates, which every V-cycle restarts from zero) and the fastest shape
// is kept.  Every shape computes the same cells with the same arithmetic:
// the choice changes the time, not the bits.
pm_status tune_rbgs(pm_batch* B) {
  static const int shapes[4][2] = {{32, 8}, {32, 4}, {16, 8}, {64, 4}};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return bfail(B, PM_ECUDA, "pm_batch: event creation failed");
  const int M = B->maxLc;
  float best = 1e30f;
  int pick = 0;
  for (int q = 0; q < 4; ++q) {
    B->rb_bx = shapes[q][0];
    B->rb_by = shapes[q][1];
    upload_vcycle_tables(B);
    float tot = 0.0f;
    for (int rep = 0; rep < 3; ++rep) {  // the first pass warms up
      cudaEventRecord(e0, B->st);
      for (int l = 0; l < M; ++l)
        for (int k = 0; k < 4; ++k) {
          BTab& t = B->t_vc[slot_down(l, k)];
          launch_rbgs_b(B->st, t.grid_max, (const RbgsDesc*)t.d_desc, t.d_tab, nullptr,
                        B->rb_bx, B->rb_by);
        }
      cudaEventRecord(e1, B->st);
      cudaEventSynchronize(e1);
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) tot += ms;
    }
    if (tot < best) {
      best = tot;
      pick = q;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  B->rb_bx = shapes[pick][0];
  B->rb_by = shapes[pick][1];
  upload_vcycle_tables(B);
  B->rb_tuned = true;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? PM_OK : bfail(B, PM_ECUDA, cudaGetErrorString(e));
}

// Capture the graph solve once (grids at their largest: the first cubes,
// which are the largest of the run): init; defect; decision; while any
// realisation is active: its V-cycle, defect and decision; the gradient
// field of each final potential.  The decision kernel sets the loop's
// condition, so no host read happens inside the solve.
pm_status build_solve_graph(pm_batch* B) {
  const int R = B->R;
  cudaError_t e = cudaSuccess;
  if (!B->st2 && (e = cudaStreamCreateWithFlags(&B->st2, cudaStreamNonBlocking)) != cudaSuccess)
    return bfail(B, PM_ECUDA, cudaGetErrorString(e));
  e = cudaStreamBeginCapture(B->st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return bfail(B, PM_ECUDA, cudaGetErrorString(e));
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  cudaGraphConditionalHandle loop = 0;
  const long long l0 = g_launches.load();
  e = cudaStreamGetCaptureInfo(B->st, &cs, nullptr, &g);
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&loop, g, 0, 0);
  auto decide = [&](cudaStream_t st) {
    launch_defect_b(st, B->t_def.grid_max, (const DefectDesc*)B->t_def.d_desc, B->t_def.d_tab,
                    B->d_active);
    launch_converged_b(st, R, B->d_scal, B->d_rel + MAX_REAL, B->d_maxv, B->d_active,
                       B->d_iters, B->d_iters + MAX_REAL, B->d_rel, loop);
  };
  cudaGraphNode_t wnode = nullptr;
  long long lb0 = 0, lb1 = 0;
  if (e == cudaSuccess) {
    launch_solve_init_b(B->st, R, B->d_active, B->d_iters, B->d_iters + MAX_REAL);
    decide(B->st);
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    e = cudaStreamGetCaptureInfo(B->st, &cs, nullptr, &g, &deps, nullptr, &nd);
    cudaGraphNodeParams p{};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = loop;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    if (e == cudaSuccess) e = cudaGraphAddNode(&wnode, g, deps, nullptr, nd, &p);
    if (e == cudaSuccess)
      e = cudaStreamUpdateCaptureDependencies(B->st, &wnode, nullptr, 1,
                                              cudaStreamSetCaptureDependencies);
    if (e == cudaSuccess) {
      cudaGraph_t body = p.conditional.phGraph_out[0];
      e = cudaStreamBeginCaptureToGraph(B->st2, body, nullptr, nullptr, 0,
                                        cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        lb0 = g_launches.load();
        launch_vcycle_slots(B, B->st2);
        decide(B->st2);
        lb1 = g_launches.load();
        e = cudaStreamEndCapture(B->st2, &body);
      }
    }
    launch_grad_b(B->st, B->t_grad.grid_max, (const GradDesc*)B->t_grad.d_desc,
                  B->t_grad.d_tab);
  }
  cudaGraph_t done = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(B->st, &done);
  // the launches counted here run when the graph does (batch_solve_done)
  g_launches.fetch_sub(g_launches.load() - l0);
  B->loop_kernels = lb1 - lb0;
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&B->sgraph, done, 0);
  if (done) cudaGraphDestroy(done);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return bfail(B, PM_ECUDA, std::string("pm_batch: solve graph: ") + cudaGetErrorString(e));
  }
  return PM_OK;
}

// The V-cycle slots in launch order, for the persistent solve.
pm_status upload_solve_slots(pm_batch* B) {
  const int M = B->maxLc, n = n_slots(M);
  if (B->d_slots && B->n_slots_dev != n) {
    cudaFree(B->d_slots);
    B->d_slots = nullptr;
  }
  if (!B->d_slots && cudaMalloc((void**)&B->d_slots, sizeof(SolveSlot) * n) != cudaSuccess)
    return bfail(B, PM_ENOMEM, "pm_batch: solve slot allocation failed");
  B->n_slots_dev = n;
  std::vector<SolveSlot> v;
  auto add = [&](int kind, int slot, int cnt) {
    v.push_back(SolveSlot{kind, cnt, B->t_vc[slot].d_desc, B->t_vc[slot].d_tab});
  };
  for (int l = 0; l < M; ++l) {
    for (int k = 0; k < 4; ++k) add(SLOT_RBGS, slot_down(l, k), 0);
    add(SLOT_RESTRICT, slot_down(l, 4), 0);
  }
  add(SLOT_CMG, slot_bottom(M), B->R);
  for (int l = M - 1; l >= 0; --l) {
    add(SLOT_PROLONG, slot_up(M, l, 0), 0);
    for (int k = 1; k < 5; ++k) add(SLOT_RBGS, slot_up(M, l, k), 0);
  }
  // synchronous: the slots change only with the V-cycle depth
  if (cudaMemcpy(B->d_slots, v.data(), sizeof(SolveSlot) * v.size(), cudaMemcpyHostToDevice) !=
      cudaSuccess)
    return bfail(B, PM_ECUDA, "pm_batch: solve slot upload failed");
  return PM_OK;
}

// The gradient-field table: every realisation's potential in buffer cur
// (alt: the other buffer, taken by the persistent solve after an odd number
// of V-cycles).
void upload_grad_table(pm_batch* B, const int* flip) {
  std::vector<GradDesc> d;
  std::vector<int> bl;
  for (int r = 0; r < B->R; ++r) {
    pm_ctx* c = B->ctx[r];
    if (c->n_active <= 0) continue;
    GradDesc e{};
    e.ph = c->phi_h[c->cur];
    e.pl = c->phi_l[c->cur];
    e.ph_alt = c->phi_h[c->cur ^ 1];
    e.pl_alt = c->phi_l[c->cur ^ 1];
    e.flip = flip;
    e.n = c->n;
    e.lo = c->lo;
    e.s = c->s;
    e.periodic = c->periodic;
    e.G = c->grad;
    set_dims(e, r, dim3((unsigned)((c->s + 31) / 32), (unsigned)((c->s + 7) / 8), (unsigned)c->s));
    d.push_back(e);
    bl.push_back(nblocks(dim3((unsigned)((c->s + 31) / 32), (unsigned)((c->s + 7) / 8),
                              (unsigned)c->s)));
  }
  tab_upload(B, B->t_grad, d, bl);
}

// The defect table of a device-decided solve: every realisation, from the
// buffer it starts in (iters: the V-cycle counts that pick the buffers in
// the graph solve; NULL for the persistent one, which keeps its own).
void upload_defect_table(pm_batch* B, const int* iters) {
  const int R = B->R;
  std::vector<DefectDesc> d;
  std::vector<int> bl;
  for (int r = 0; r < R; ++r) {
    pm_ctx* c = B->ctx[r];
    const int lo = c->lo, s = c->s, c0 = c->cur;
    DefectDesc e{};
    e.ph = full_view(c, c->phi_h[c0], lo, s);
    e.pl = full_view(c, c->phi_l[c0], lo, s);
    e.qh = full_view(c, c->phi_h[c0 ^ 1], lo, s);
    e.ql = full_view(c, c->phi_l[c0 ^ 1], lo, s);
    e.e = compact_view(c->lu[0], s);
    e.fh = full_view(c, c->f_hi, lo, s);
    e.fl = full_view(c, c->f_lo, lo, s);
    e.rb = compact_view(c->lb[0], s);
    e.periodic = c->periodic;
    e.write_r = 1;
    e.partial = c->partial;
    e.counter = c->counter;
    e.out = B->d_scal + 16 * r + 11;
    e.iters = iters;
    set_dims(e, r, defect_grid(s));
    d.push_back(e);
    bl.push_back(nblocks(defect_grid(s)));
  }
  tab_upload(B, B->t_def, d, bl);
}

// One persistent launch solves every realisation from its current buffer to
// its tolerance; V-cycle counts, failures and residuals are read back when
// the step ends (batch_solve_done).
pm_status batch_solve_persistent(pm_batch* B) {
  const int R = B->R;
  if (B->tables_stale) {
    upload_vcycle_tables(B);
    B->tables_stale = false;
  }
  if (!B->d_slots || B->n_slots_dev != n_slots(B->maxLc)) {
    pm_status st = upload_solve_slots(B);
    if (st != PM_OK) return st;
  }
  upload_defect_table(B, nullptr);
  upload_grad_table(B, nullptr);
  cudaMemsetAsync(B->d_bar, 0, sizeof(GridBar), B->st);
  cudaMemsetAsync(B->d_iters + MAX_REAL, 0, sizeof(int) * R, B->st);
  SolveArgs a{};
  a.grad = (const GradDesc*)B->t_grad.d_desc;
  a.grad_t = B->t_grad.d_tab;
  a.def = (const DefectDesc*)B->t_def.d_desc;
  a.def_t = B->t_def.d_tab;
  a.slots = B->d_slots;
  a.n_slots = B->n_slots_dev;
  a.R = R;
  a.scal = B->d_scal;
  a.rtol = B->d_rel + MAX_REAL;
  a.maxv = B->d_maxv;
  a.iters = B->d_iters;
  a.failed = B->d_iters + MAX_REAL;
  a.rel = B->d_rel;
  a.bar = B->d_bar;
  a.limit_ns = (unsigned long long)(B->wait_s * 1e9);
  a.extra = B->extra;
  a.fast_coarse = cmg_fast();
  cudaError_t e = launch_solve_b(B->st, a);
  if (e != cudaSuccess) return bfail(B, PM_ECUDA, cudaGetErrorString(e));
  B->solved_on_device = true;
  return PM_OK;
}

// One launch of the solve graph (captured at the first solve).
pm_status batch_solve_graph(pm_batch* B) {
  if (B->tables_stale) {
    upload_vcycle_tables(B);
    B->tables_stale = false;
  }
  if (!B->rb_tuned) {
    pm_status st = tune_rbgs(B);
    if (st != PM_OK) return st;
  }
  upload_defect_table(B, B->d_iters);
  upload_grad_table(B, B->d_iters);
  if (!B->sgraph) {
    pm_status st = build_solve_graph(B);
    if (st != PM_OK) return st;
  }
  cudaError_t e = cudaGraphLaunch(B->sgraph, B->st);
  if (e != cudaSuccess) return bfail(B, PM_ECUDA, cudaGetErrorString(e));
  B->solved_on_device = true;
  return PM_OK;
}

pm_status batch_sync(pm_batch* B) {
  if (B->solved_on_device) {
    cudaMemcpyAsync(B->h_iters, B->d_iters, sizeof(int) * 2 * MAX_REAL, cudaMemcpyDeviceToHost,
                    B->st);
    cudaMemcpyAsync(B->h_rel, B->d_rel, sizeof(double) * B->R, cudaMemcpyDeviceToHost, B->st);
    cudaMemcpyAsync(B->h_bar, B->d_bar, sizeof(GridBar), cudaMemcpyDeviceToHost, B->st);
  }
  cudaMemcpyAsync(B->h_scal, B->d_scal, sizeof(double) * 16 * B->R, cudaMemcpyDeviceToHost,
                  B->st);
  cudaMemcpyAsync(B->h_cnt, B->d_cnt, sizeof(unsigned long long) * 4 * B->R,
                  cudaMemcpyDeviceToHost, B->st);
  cudaError_t e = cudaStreamSynchronize(B->st);
  if (e != cudaSuccess) return bfail(B, PM_ECUDA, cudaGetErrorString(e));
  e = cudaGetLastError();
  if (e != cudaSuccess) return bfail(B, PM_ECUDA, cudaGetErrorString(e));
  return PM_OK;
}

// After the step's sync: the outcome of a persistent solve per realisation
// (its potential ends in the buffer of parity iters relative to the start).
pm_status batch_solve_done(pm_batch* B) {
  if (!B->solved_on_device) return PM_OK;
  B->solved_on_device = false;
  if (B->h_bar->err) {
    char buf[200];
    snprintf(buf, sizeof buf,
             "pm_batch_step: a grid barrier of the persistent solve waited longer than %.3g s "
             "(pass %d); the batch must be destroyed",
             B->wait_s, B->h_bar->where);
    return bfail(B, PM_ETIMEOUT, buf);
  }
  if (!B->persistent) {
    // the graph's kernels: init, defect, decision, gradient, and the loop's
    // body once per V-cycle of the realisation that took the most
    int most = 0;
    for (int r = 0; r < B->R; ++r) most = std::max(most, B->h_iters[r]);
    g_launches.fetch_add(4 + (long long)most * B->loop_kernels);
  }
  for (int r = 0; r < B->R; ++r) {
    pm_ctx* c = B->ctx[r];
    const int it = B->h_iters[r];
    if (B->h_iters[MAX_REAL + r]) {
      char buf[200];
      snprintf(buf, sizeof buf,
               "realisation %d: relative residual %.3e after %d V-cycles (rtol %.1e)", r,
               B->h_rel[r], it, c->cfg.rtol);
      return bfail(B, PM_ENOCONV, buf);
    }
    c->cur ^= it & 1;
    c->vcycles_last = it;
    c->vcycles_total += it;
    c->resid_last = B->h_rel[r];
  }
  return PM_OK;
}

}  // namespace

extern "C" {

pm_status pm_batch_init(int32_t n_real, const pm_config* cfgs, const float* const* pos4,
                        const float* const* mom4, int32_t host_mem, void* stream,
                        pm_batch** out) {
  if (!out) return bfail(nullptr, PM_EINVAL, "pm_batch_init: out is NULL");
  *out = nullptr;
  if (n_real < 1 || n_real > MAX_REAL || !cfgs || !pos4 || !mom4 || !stream)
    return bfail(nullptr, PM_EINVAL, "pm_batch_init: bad argument");
  for (int r = 0; r < n_real; ++r) {
    if (cfgs[r].precision != PM_MIXED)
      return bfail(nullptr, PM_EINVAL, "pm_batch_init: batches run in PM_MIXED precision");
    if (cfgs[r].guess == PM_GUESS_LEARNED)
      return bfail(nullptr, PM_EINVAL, "pm_batch_init: the learned guess runs per context");
    if (cfgs[r].gravity != PM_GRAVITY_POISSON)
      return bfail(nullptr, PM_EINVAL, "pm_batch_init: batches solve Poisson's equation");
    if (cfgs[r].domain != PM_DOMAIN_CUBE)
      return bfail(nullptr, PM_EINVAL, "pm_batch_init: batches keep a cube");
    if (cfgs[r].assignment != PM_ASSIGN_CIC)
      return bfail(nullptr, PM_EINVAL, "pm_batch_init: batches assign by CIC");
    if (cfgs[r].shrink == PM_SHRINK_RECORD)
      return bfail(nullptr, PM_EINVAL, "pm_batch_init: the fixed-box lightcone record runs "
                                       "per context");
    if (cfgs[r].inner_vcycles > 1)
      return bfail(nullptr, PM_EINVAL, "pm_batch_init: batches run one V-cycle per defect "
                                       "(inner_vcycles <= 1)");
    if (cfgs[r].sort_every != 0)
      return bfail(nullptr, PM_EINVAL, "pm_batch_init: the particle order by cell runs "
                                       "per context (sort_every = 0)");
    if (cfgs[r].n_steps != cfgs[0].n_steps || cfgs[r].a_init != cfgs[0].a_init ||
        cfgs[r].a_final != cfgs[0].a_final)
      return bfail(nullptr, PM_EINVAL, "pm_batch_init: realisations must share the a schedule");
  }
  pm_batch* B = new pm_batch();
  B->R = n_real;
  B->st = (cudaStream_t)stream;
  for (int r = 0; r < n_real; ++r) {
    pm_ctx* c = nullptr;
    pm_status s = pm_init(&cfgs[r], pos4[r], mom4[r], host_mem, stream, &c);
    if (s != PM_OK) {
      B->err = std::string("pm_batch_init: realisation ") + std::to_string(r) + ": " + g_err;
      g_err = B->err;
      pm_batch_destroy(B);
      return s;
    }
    c->use_graphs = false;
    B->ctx.push_back(c);
  }
  pm_status st = PM_OK;
  if (cudaMalloc((void**)&B->d_active, sizeof(int) * MAX_REAL) != cudaSuccess ||
      cudaMalloc((void**)&B->d_scal, sizeof(double) * 16 * MAX_REAL) != cudaSuccess ||
      cudaMallocHost((void**)&B->h_scal, sizeof(double) * 16 * MAX_REAL) != cudaSuccess ||
      cudaMalloc((void**)&B->d_cnt, sizeof(unsigned long long) * 4 * MAX_REAL) != cudaSuccess ||
      cudaMallocHost((void**)&B->h_cnt, sizeof(unsigned long long) * 4 * MAX_REAL) !=
          cudaSuccess ||
      cudaMalloc((void**)&B->d_ovf, sizeof(int) * MAX_REAL) != cudaSuccess ||
      cudaMalloc((void**)&B->d_bar, sizeof(GridBar)) != cudaSuccess ||
      cudaMallocHost((void**)&B->h_bar, sizeof(GridBar)) != cudaSuccess ||
      cudaMalloc((void**)&B->d_iters, sizeof(int) * 2 * MAX_REAL) != cudaSuccess ||
      cudaMallocHost((void**)&B->h_iters, sizeof(int) * 2 * MAX_REAL) != cudaSuccess ||
      cudaMalloc((void**)&B->d_rel, sizeof(double) * 2 * MAX_REAL) != cudaSuccess ||
      cudaMallocHost((void**)&B->h_rel, sizeof(double) * MAX_REAL) != cudaSuccess ||
      cudaMalloc((void**)&B->d_maxv, sizeof(int) * MAX_REAL) != cudaSuccess)
    st = bfail(B, PM_ENOMEM, "pm_batch_init: allocation failed");
  if (st == PM_OK) {
    // per-realisation tolerances of the persistent solve (fixed for the run)
    double tol[MAX_REAL];
    int mv[MAX_REAL];
    for (int r = 0; r < n_real; ++r) {
      tol[r] = cfgs[r].rtol;
      mv[r] = cfgs[r].max_vcycles;
    }
    if (cudaMemcpy(B->d_rel + MAX_REAL, tol, sizeof(double) * n_real, cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(B->d_maxv, mv, sizeof(int) * n_real, cudaMemcpyHostToDevice) != cudaSuccess)
      st = bfail(B, PM_ECUDA, "pm_batch_init: tolerance upload failed");
    // the graph solve by default (measured faster than the persistent
    // kernel, whose register budget is that of its heaviest phase)
    B->persistent = false;
  }
  if (st == PM_OK) st = tab_alloc(B, B->t_dep, sizeof(DepositDesc));
  if (st == PM_OK) st = tab_alloc(B, B->t_src, sizeof(SourceDesc));
  if (st == PM_OK) st = tab_alloc(B, B->t_bnd, sizeof(BoundaryDesc));
  if (st == PM_OK) st = tab_alloc(B, B->t_pred, sizeof(PredictDesc));
  if (st == PM_OK) st = tab_alloc(B, B->t_def, sizeof(DefectDesc));
  if (st == PM_OK) st = tab_alloc(B, B->t_grad, sizeof(GradDesc));
  if (st == PM_OK) st = tab_alloc(B, B->t_gat, sizeof(GatherDesc));
  if (st == PM_OK) st = tab_alloc(B, B->t_scan, sizeof(ScanDesc));
  if (st == PM_OK) st = tab_alloc(B, B->t_scat, sizeof(ScatterDesc));
  if (st != PM_OK) {
    pm_batch_destroy(B);
    return st;
  }
  cudaMemsetAsync(B->d_scal, 0, sizeof(double) * 16 * MAX_REAL, B->st);
  cudaMemsetAsync(B->d_cnt, 0, sizeof(unsigned long long) * 4 * MAX_REAL, B->st);
  cudaMemsetAsync(B->d_ovf, 0, sizeof(int) * MAX_REAL, B->st);
  cudaMemsetAsync(B->d_iters, 0, sizeof(int) * 2 * MAX_REAL, B->st);
  *out = B;
  return PM_OK;
}

pm_status pm_batch_step(pm_batch* B, int32_t n_steps) {
  if (!B) return bfail(nullptr, PM_EINVAL, "pm_batch_step: NULL batch");
  const int R = B->R;
  for (int q = 0; q < n_steps; ++q) {
    const int k = B->ctx[0]->step;
    if (k >= B->ctx[0]->cfg.n_steps) return bfail(B, PM_EINVAL, "pm_batch_step: past the end");
    // per realisation: active cube, phase, schedule scalars
    std::vector<int> phase_changed(R, 0);
    for (int r = 0; r < R; ++r) {
      pm_ctx* c = B->ctx[r];
      int lo, s, per;
      geometry(c, c->R[k], &lo, &s, &per);
      phase_changed[r] = !c->cube_valid || per != c->periodic;
      bool changed = !c->cube_valid || lo != c->lo || s != c->s || per != c->periodic;
      pm_status st = set_cube(c, lo, s, per, c->R[k]);
      if (st != PM_OK) return bfail(B, st, c->err);
      if (changed) B->tables_stale = true;
    }
    if (B->t_vc.empty()) {
      // the first configuration fixes the V-cycle depth (cubes only shrink)
      int M = 0;
      for (int r = 0; r < R; ++r) M = std::max(M, first_small_level(B->ctx[r]));
      B->maxLc = M;
      B->t_vc.resize(n_slots(M));
      for (auto& t : B->t_vc) {
        size_t sz = std::max(std::max(sizeof(RbgsDesc), sizeof(RestrictDesc)),
                             std::max(sizeof(ProlongDesc), sizeof(CmgDesc)));
        pm_status st = tab_alloc(B, t, sz);
        if (st != PM_OK) return st;
      }
    }
    // 1-2. half drift + deposit
    {
      std::vector<DepositDesc> d;
      std::vector<int> bl;
      for (int r = 0; r < R; ++r) {
        pm_ctx* c = B->ctx[r];
        if (c->n_active <= 0) continue;
        DepositDesc e{};
        e.pos = c->pos;
        e.mom = c->mom;
        e.N = c->n_active;
        e.c0 = (float)(c->dtau[k] / (2.0 * c->a[k]));
        e.n = c->n;
        e.lo = c->lo;
        e.s = c->s;
        e.periodic = c->periodic;
        e.rho = c->rho;
        e.escaped = c->d_cnt + 1;
        int nb = deposit_blocks(c->n_active);
        set_dims(e, r, dim3(nb, 1, 1));
        d.push_back(e);
        bl.push_back(nb);
      }
      int g = tab_upload(B, B->t_dep, d, bl);
      launch_deposit_b(B->st, g, (const DepositDesc*)B->t_dep.d_desc, B->t_dep.d_tab);
    }
    // 3. source (+ moments), boundary ghosts in both potential buffers, predict
    {
      std::vector<SourceDesc> d;
      std::vector<int> bl;
      for (int r = 0; r < R; ++r) {
        pm_ctx* c = B->ctx[r];
        const int n = c->n, lo = c->lo, s = c->s;
        const double S = 1.5 * c->cfg.omega_m / c->a_half[k];
        const double nbar = (double)c->N0 / ((double)n * n * n);
        const double invM = 1.0 / (281474976710656.0 * nbar);
        SourceDesc e{};
        e.rho = c->rho;
        e.n = n;
        e.lo = lo;
        e.s = s;
        e.fh = full_view(c, c->f_hi, lo, s);
        e.fl = full_view(c, c->f_lo, lo, s);
        e.invM.hi = (float)invM;
        e.invM.lo = (float)(invM - (double)e.invM.hi);
        e.S.hi = (float)S;
        e.S.lo = (float)(S - (double)e.S.hi);
        e.bgw = c->bgw;
        e.moments = !c->periodic;
        e.partial_f2 = c->partial;
        e.partial_m = c->partial_m;
        e.counter = c->counter;
        e.out = B->d_scal + 16 * r;
        e.bgm = c->bgm;
        e.invM_d = invM;
        e.overflow = B->d_ovf + r;
        set_dims(e, r, source_grid(s));
        d.push_back(e);
        bl.push_back(nblocks(source_grid(s)));
      }
      int g = tab_upload(B, B->t_src, d, bl);
      launch_source_b(B->st, g, (const SourceDesc*)B->t_src.d_desc, B->t_src.d_tab);
    }
    {
      std::vector<BoundaryDesc> d;
      std::vector<int> bl;
      for (int r = 0; r < R; ++r) {
        pm_ctx* c = B->ctx[r];
        if (c->periodic) continue;
        for (int qb = 0; qb < 2; ++qb) {
          BoundaryDesc e{};
          e.ph = full_view(c, c->phi_h[qb], c->lo, c->s);
          e.pl = full_view(c, c->phi_l[qb], c->lo, c->s);
          e.n = c->n;
          e.lo = c->lo;
          e.mom = B->d_scal + 16 * r + 1;
          e.S = 1.5 * c->cfg.omega_m / c->a_half[k];
          e.want_lo = 1;
          int nb = boundary_blocks(c->s);
          set_dims(e, r, dim3(nb, 1, 1));
          d.push_back(e);
          bl.push_back(nb);
        }
      }
      int g = tab_upload(B, B->t_bnd, d, bl);
      launch_boundary_b(B->st, g, (const BoundaryDesc*)B->t_bnd.d_desc, B->t_bnd.d_tab);
    }
    {
      std::vector<PredictDesc> d;
      std::vector<int> bl;
      for (int r = 0; r < R; ++r) {
        pm_ctx* c = B->ctx[r];
        if (c->cfg.guess != PM_GUESS_WARM) continue;
        if (phase_changed[r]) c->n_sol = 0;
        if (c->n_sol < 1) continue;
        float w = 0.0f;
        if (c->n_sol >= 2) {
          double d0 = c->ah_hist[1] - c->ah_hist[0];
          w = d0 > 0 ? (float)((c->a_half[k] - c->ah_hist[1]) / d0) : 0.0f;
        }
        PredictDesc e{};
        e.ph = full_view(c, c->phi_h[c->cur], c->lo, c->s);
        e.pl = full_view(c, c->phi_l[c->cur], c->lo, c->s);
        e.qh = full_view(c, c->prev_hi, c->lo, c->s);
        e.ql = full_view(c, c->prev_lo, c->lo, c->s);
        e.w = w;
        e.pair = 1;
        set_dims(e, r, full_grid_b(c->s));
        d.push_back(e);
        bl.push_back(nblocks(full_grid_b(c->s)));
      }
      int g = tab_upload(B, B->t_pred, d, bl);
      launch_predict_b(B->st, g, (const PredictDesc*)B->t_pred.d_desc, B->t_pred.d_tab);
    }
    // 4. solve every realisation to its rtol, decided on the device
    {
      pm_status st = B->persistent ? batch_solve_persistent(B) : batch_solve_graph(B);
      if (st != PM_OK) return st;
    }
    for (int r = 0; r < R; ++r) {
      pm_ctx* c = B->ctx[r];
      c->ah_hist[0] = c->ah_hist[1];
      c->ah_hist[1] = c->a_half[k];
      c->n_sol++;
    }
    // 5-6. gather + kick + drift (+ keep flags) from the gradient field the
    // solve wrote
    bool any_flag = false;
    std::vector<int> flagged(R, 0);
    {
      std::vector<GatherDesc> d;
      std::vector<int> bl;
      for (int r = 0; r < R; ++r) {
        pm_ctx* c = B->ctx[r];
        if (c->n_active <= 0) continue;
        const double R1 = c->R[k + 1];
        const bool do_flag =
            c->cfg.shrink == PM_SHRINK_ON && c->cfg.bc != PM_BC_PERIODIC && is_open(c, R1);
        GatherDesc e{};
        e.pos = c->pos;
        e.mom = c->mom;
        e.N = c->n_active;
        e.G = c->grad;
        e.n = c->n;
        e.lo = c->lo;
        e.s = c->s;
        e.periodic = c->periodic;
        e.kick = (float)(c->a_half[k] * c->dtau[k]);
        e.c2 = (float)(c->dtau[k] / (2.0 * c->a[k + 1]));
        e.do_flag = do_flag;
        if (do_flag) keep_bounds(0.5 * c->n, R1, &e.klo, &e.khi);
        e.flags = c->flags;
        e.block_keep = c->block_keep;
        e.forces = c->forces;  // NULL unless the realisation stores forces
        e.escaped = c->d_cnt + 1;
        c->forces_valid = c->forces != nullptr;
        c->forces_n = c->n_active;
        int nb = gkd_blocks(c->n_active);
        set_dims(e, r, dim3(nb, 1, 1));
        d.push_back(e);
        bl.push_back(nb);
        flagged[r] = do_flag;
        any_flag |= do_flag;
      }
      int g = tab_upload(B, B->t_gat, d, bl);
      launch_gather_b(B->st, g, (const GatherDesc*)B->t_gat.d_desc, B->t_gat.d_tab);
    }
    // 7. lightcone shrink of the flagged realisations
    if (any_flag) {
      std::vector<ScanDesc> ds;
      std::vector<ScatterDesc> dc;
      std::vector<int> bs, bc;
      for (int r = 0; r < R; ++r) {
        if (!flagged[r]) continue;
        pm_ctx* c = B->ctx[r];
        const int nb = gkd_blocks(c->n_active);
        ScanDesc e{};
        e.cnt = c->block_keep;
        e.off = c->keep_off;
        e.nblk = nb;
        e.n_keep = B->d_cnt + 4 * r;
        set_dims(e, r, dim3(1, 1, 1));
        ds.push_back(e);
        bs.push_back(1);
        ScatterDesc f{};
        f.pos = c->pos;
        f.mom = c->mom;
        f.N = c->n_active;
        f.flags = c->flags;
        f.keep_off = c->keep_off;
        f.pos_out = c->pos2;
        f.mom_out = c->mom2;
        f.lc_pos = c->lc_pos;
        f.lc_mom = c->lc_mom;
        f.lc_base = c->n_lc;
        f.a_cross = (float)c->a[k + 1];
        set_dims(f, r, dim3(nb, 1, 1));
        dc.push_back(f);
        bc.push_back(nb);
      }
      int g = tab_upload(B, B->t_scan, ds, bs);
      launch_scan_b(B->st, g, (const ScanDesc*)B->t_scan.d_desc, B->t_scan.d_tab);
      g = tab_upload(B, B->t_scat, dc, bc);
      launch_scatter_b(B->st, g, (const ScatterDesc*)B->t_scat.d_desc, B->t_scat.d_tab);
    }
    pm_status st = batch_sync(B);
    if (st != PM_OK) return st;
    st = batch_solve_done(B);
    if (st != PM_OK) return st;
    for (int r = 0; r < R; ++r) {
      pm_ctx* c = B->ctx[r];
      c->particle_steps += c->n_active;
      if (flagged[r]) {
        long long keep = (long long)B->h_cnt[4 * r];
        std::swap(c->pos, c->pos2);
        std::swap(c->mom, c->mom2);
        c->n_lc += c->n_active - keep;
        c->n_active = keep;
      }
      c->step++;
    }
    int ovf[MAX_REAL];
    if (cudaMemcpy(ovf, B->d_ovf, sizeof(int) * R, cudaMemcpyDeviceToHost) != cudaSuccess)
      return bfail(B, PM_ECUDA, "pm_batch_step: reading the overflow flags");
    for (int r = 0; r < R; ++r)
      if (ovf[r]) return bfail(B, PM_EOVERFLOW, "deposit: a cell count exceeded 2^62");
  }
  return PM_OK;
}

pm_status pm_batch_stats(pm_batch* B, int32_t r, pm_stats_t* out) {
  if (!B || r < 0 || r >= B->R) return bfail(B, PM_EINVAL, "pm_batch_stats: bad argument");
  return pm_stats(B->ctx[r], out);
}

pm_status pm_batch_get_forces(pm_batch* B, int32_t r, float* f4, int32_t host_mem,
                              int64_t* n_out) {
  if (!B || r < 0 || r >= B->R) return bfail(B, PM_EINVAL, "pm_batch_get_forces: bad argument");
  pm_status st = pm_get_forces(B->ctx[r], f4, host_mem, n_out);
  if (st != PM_OK) B->err = B->ctx[r]->err;
  return st;
}

pm_status pm_batch_get_particles(pm_batch* B, int32_t r, float* pos4, float* mom4,
                                 int32_t host_mem, int64_t* n_active_out) {
  if (!B || r < 0 || r >= B->R) return bfail(B, PM_EINVAL, "pm_batch_get_particles");
  return pm_get_particles(B->ctx[r], pos4, mom4, host_mem, n_active_out);
}

pm_status pm_batch_get_lightcone(pm_batch* B, int32_t r, float* pos4, float* mom4,
                                 int32_t host_mem, int64_t* n_out) {
  if (!B || r < 0 || r >= B->R) return bfail(B, PM_EINVAL, "pm_batch_get_lightcone");
  return pm_get_lightcone(B->ctx[r], pos4, mom4, host_mem, n_out);
}

pm_status pm_batch_set_solve(pm_batch* B, int32_t persistent, double wait_seconds,
                             int32_t extra_arrivals) {
  if (!B) return bfail(nullptr, PM_EINVAL, "pm_batch_set_solve: NULL batch");
  if (!(wait_seconds > 0.0) || !std::isfinite(wait_seconds) || wait_seconds > 3600.0 ||
      extra_arrivals < 0 || (persistent != 0 && persistent != 1))
    return bfail(B, PM_EINVAL, "pm_batch_set_solve: bad argument");
  if (persistent && !(cmg_cluster() == 1 && solve_grid_b() > 0))
    return bfail(B, PM_EINVAL, "pm_batch_set_solve: the persistent solve cannot run here "
                               "(coarse levels in a cluster, or grid not resident)");
  if (persistent != (int)B->persistent) {
    B->persistent = persistent != 0;
    // block shape of the colour pass: the persistent kernel's, or autotuned
    B->rb_bx = 32;
    B->rb_by = 8;
    B->rb_tuned = B->persistent;
    B->tables_stale = true;
    if (B->sgraph) {
      cudaStreamSynchronize(B->st);
      cudaGraphExecDestroy(B->sgraph);
      B->sgraph = nullptr;
    }
  }
  B->wait_s = wait_seconds;
  B->extra = extra_arrivals;
  return PM_OK;
}

const char* pm_batch_last_error(const pm_batch* B) { return B ? B->err.c_str() : g_err.c_str(); }

void pm_batch_destroy(pm_batch* B) {
  if (!B) return;
  if (B->st) cudaStreamSynchronize(B->st);
  if (B->sgraph) cudaGraphExecDestroy(B->sgraph);
  if (B->st2) cudaStreamDestroy(B->st2);
  for (pm_ctx* c : B->ctx) pm_destroy(c);
  for (BTab* t : {&B->t_dep, &B->t_src, &B->t_bnd, &B->t_pred, &B->t_def, &B->t_grad,
                  &B->t_gat, &B->t_scan, &B->t_scat})
    tab_free(*t);
  for (auto& t : B->t_vc) tab_free(t);
  if (B->d_active) cudaFree(B->d_active);
  if (B->d_bar) cudaFree(B->d_bar);
  if (B->h_bar) cudaFreeHost(B->h_bar);
  if (B->d_iters) cudaFree(B->d_iters);
  if (B->h_iters) cudaFreeHost(B->h_iters);
  if (B->d_rel) cudaFree(B->d_rel);
  if (B->h_rel) cudaFreeHost(B->h_rel);
  if (B->d_maxv) cudaFree(B->d_maxv);
  if (B->d_slots) cudaFree(B->d_slots);
  if (B->d_scal) cudaFree(B->d_scal);
  if (B->h_scal) cudaFreeHost(B->h_scal);
  if (B->d_cnt) cudaFree(B->d_cnt);
  if (B->h_cnt) cudaFreeHost(B->h_cnt);
  if (B->d_ovf) cudaFree(B->d_ovf);
  delete B;
}

}  // extern "C"

// ===========================================================================
// Tensor-core building blocks of the learned guess
// ===========================================================================
namespace {
Grid padded_view(const float* base, int s) {
  Grid g{};
  g.s = s;
  g.sy = s + 2;
  g.sz = (s + 2) * (s + 2);
  g.base = const_cast<float*>(base) + 1 + g.sy + g.sz;
  return g;
}
pm_status finish_test_call(cudaStream_t st) {
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(nullptr, PM_ECUDA, cudaGetErrorString(e));
  return PM_OK;
}
}  // namespace

extern "C" pm_status pm_mg_restrict(const float* u, const float* b, int32_t s, int32_t periodic,
                                    float h2, float gam, float* uc, float* bc, void* stream) {
  if (!u || !b || !uc || !bc || s < 4 || (s & 1) || s > 2048 || !(h2 > 0))
    return fail(nullptr, PM_EINVAL, "pm_mg_restrict: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  launch_resid_restrict(st, padded_view(u, s), padded_view(b, s), 1.0f / h2,
                        padded_view(uc, s / 2), padded_view(bc, s / 2), periodic, gam);
  return finish_test_call(st);
}

extern "C" pm_status pm_mg_prolong(const float* uc, float* u, int32_t s, int32_t periodic,
                                   float gam_c, void* stream) {
  if (!u || !uc || s < 4 || (s & 1) || s > 2048)
    return fail(nullptr, PM_EINVAL, "pm_mg_prolong: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  launch_prolong(st, padded_view(uc, s / 2), padded_view(u, s), periodic, gam_c);
  return finish_test_call(st);
}

extern "C" pm_status pm_mg_smooth(const float* u_in, float* u_out, const float* b, int32_t s,
                                  int32_t periodic, float h2, float gam, int32_t zero_start,
                                  int32_t fused, int32_t zchunk, void* stream) {
  if (!u_out || !b || (!u_in && !zero_start) || s < 4 || (s & 1) || s > 2048 || zchunk < 0 ||
      (fused != 0 && fused != 1 && !rbgs2_tile_ok(fused)) ||
      (fused && !zero_start && u_in == u_out))
    return fail(nullptr, PM_EINVAL, "pm_mg_smooth: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  if (mg_prepare() != cudaSuccess) return fail(nullptr, PM_ECUDA, "pm_mg_smooth: attributes");
  auto view = [&](const float* base) {
    Grid g{};
    g.s = s;
    g.sy = s + 2;
    g.sz = (s + 2) * (s + 2);
    g.base = const_cast<float*>(base) + 1 + g.sy + g.sz;
    return g;
  };
  Grid wi = view(u_in ? u_in : u_out), wo = view(u_out), gb = view(b);
  if (fused) {
    launch_rbgs2(st, wi, wo, gb, h2, periodic, gam, zero_start != 0, zchunk, 6.0f,
                 fused == 1 ? 16 : fused);
  } else {
    const size_t bytes = sizeof(float) * (size_t)(s + 2) * (s + 2) * (s + 2);
    if (zero_start && cudaMemsetAsync(u_out, 0, bytes, st) != cudaSuccess)
      return fail(nullptr, PM_ECUDA, "pm_mg_smooth: clear");
    if (!zero_start && u_in != u_out &&
        cudaMemcpyAsync(u_out, u_in, bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return fail(nullptr, PM_ECUDA, "pm_mg_smooth: copy");
    for (int sw = 0; sw < 2; ++sw) {
      launch_rbgs(st, wo, gb, h2, 0, periodic, gam, zero_start && sw == 0 ? 1 : 0);
      launch_rbgs(st, wo, gb, h2, 1, periodic, gam, zero_start && sw == 0 ? 2 : 0);
    }
  }
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(nullptr, PM_ECUDA, cudaGetErrorString(e));
  return PM_OK;
}

extern "C" pm_status pm_selftest_wait(int32_t arrive, int64_t polls, void* stream) {
  if (polls < 1 || polls > 1000000000LL)
    return fail(nullptr, PM_EINVAL, "pm_selftest_wait: polls in [1, 1e9]");
  cudaStream_t st = (cudaStream_t)stream;
  int* flag = nullptr;
  if (cudaMallocAsync((void**)&flag, sizeof(int), st) != cudaSuccess)
    return fail(nullptr, PM_ENOMEM, "pm_selftest_wait: cudaMallocAsync");
  cudaMemsetAsync(flag, 0, sizeof(int), st);
  launch_wait_selftest(st, arrive ? 1 : 0, polls, flag);
  cudaError_t e = cudaGetLastError();
  int h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFreeAsync(flag, st);
  if (e != cudaSuccess) return fail(nullptr, PM_ECUDA, cudaGetErrorString(e));
  if (h) return fail(nullptr, PM_ETIMEOUT, "pm_selftest_wait: the bounded wait gave up");
  return PM_OK;
}

extern "C" pm_status pm_nn_gemm_bf16(const void* A, const void* B, float* C, int32_t M,
                                     int32_t N, int32_t K, void* stream) {
  if (!A || !B || !C || M <= 0 || M % 128 || K <= 0 || K % 64 ||
      (N != 16 && N != 32 && N != 64 && N != 128))
    return fail(nullptr, PM_EINVAL, "pm_nn_gemm_bf16: M % 128, K % 64, N in {16,32,64,128}");
  cudaStream_t st = (cudaStream_t)stream;
  int* err = nullptr;
  if (cudaMallocAsync((void**)&err, sizeof(int), st) != cudaSuccess)
    return fail(nullptr, PM_ENOMEM, "pm_nn_gemm_bf16: cudaMallocAsync");
  cudaMemsetAsync(err, 0, sizeof(int), st);
  launch_gemm_tc(st, A, B, C, M, N, K, err);
  cudaError_t e = cudaGetLastError();
  int h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFreeAsync(err, st);
  if (e != cudaSuccess) return fail(nullptr, PM_ECUDA, cudaGetErrorString(e));
  if (h) return fail(nullptr, PM_ETIMEOUT, "pm_nn_gemm_bf16: MMA completion wait timed out");
  return PM_OK;
}
