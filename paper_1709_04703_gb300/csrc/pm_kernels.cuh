// Host-side launchers of the libpmshrink kernels (one stream each).
#pragma once

#include "pm_common.cuh"

namespace pm {

// Counts kernel launches made by the library (pm_launch_count).
void note_launch();

// Launch with the programmatic-stream-serialization attribute (the kernel
// starts with pdl_wait); a normal launch when PM_NO_PDL is set.
bool pdl_enabled();
template <typename... Exp, typename... Act>
void launch_pdl(void (*k)(Exp...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                Act&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  cudaLaunchKernelEx(&cfg, k, static_cast<Exp>(args)...);
}

// pm_shrink's keep rule: R = chi(a)/cell + buffer (cells), and the exact
// float bounds of |x - n/2| <= R (everything kept while R > n/2 - 1).
double shrink_radius_cells(int n, double box, double om, double ol, double buffer, double a);
void shrink_keep_bounds(int n, double R, float* klo, float* khi);

// k_sort.cu: stable radix sort of the particles by the cell of their CIC
// base node (keys: ((z n + y) n + x) of floor(u - 1/2) wrapped into [0, n))
struct SortWork {
  unsigned* keys[2];  // N each
  unsigned* vals[2];  // N each
  unsigned* counts;   // sort_counts_len(N)
  unsigned* ghist;    // sort_ghist_len()
};
int sort_passes(int n);
size_t sort_counts_len(long long N);
size_t sort_ghist_len();
// pos_out/mom_out <- pos/mom in the sorted order (must not alias them)
cudaError_t launch_sort_particles(cudaStream_t st, const float4* pos, const float4* mom,
                                  long long N, int n, const SortWork& w, float4* pos_out,
                                  float4* mom_out);

// k_fp64.cu: the Poisson V-cycle and defect in double (PM_FP64_PLAIN)
void launch64_rbgs(cudaStream_t st, GridD u, GridD b, double h2, int color, int periodic,
                   double gam);
void launch64_resid_restrict(cudaStream_t st, GridD u, GridD b, double inv_h2, GridD uc,
                             GridD bc, int periodic, double gam);
void launch64_prolong(cudaStream_t st, GridD uc, GridD u, int periodic, double gam_c);
void launch64_bottom(cudaStream_t st, GridD u, GridD b, double h2, int periodic, double gam,
                     int sweeps);
int defect64_blocks(int s);
void launch64_defect(cudaStream_t st, GridD p, GridD f, int periodic, double* partial,
                     unsigned int* counter, double* out);
void launch64_from_pair(cudaStream_t st, Grid hi, Grid lo, GridD out, bool ghost);
void launch64_to_pair(cudaStream_t st, GridD in, Grid hi, Grid lo, bool ghost);
// mixed precision with an FP64 outer loop (PM_MIXED_FP64)
void launch64_correct(cudaStream_t st, GridD p, Grid e);
void launch64m_defect(cudaStream_t st, GridD p, GridD f, Grid rb, int periodic, double* partial,
                      unsigned int* counter, double* out);
void launch64_predict(cudaStream_t st, GridD p, GridD q, double w);
void launch64_fill(cudaStream_t st, GridD p, double v);
void launch64_grad(cudaStream_t st, const double* ph, int n, int lo, int s, int periodic,
                   float4* G);
void launch_boundary64(cudaStream_t st, GridD p, int n, int lo, const double* mom, double S);

// k_mesh.cu
void launch_drift_deposit(cudaStream_t st, int grid, float4* pos, const float4* mom,
                          long long N, float c0, bool drift, int n, int lo, int s,
                          int periodic, unsigned long long* rho,
                          unsigned long long* escaped);
void launch_source(cudaStream_t st, int grid, unsigned long long* rho, int n, int lo,
                   int s, Grid fh, Grid fl, double invM, double S, const df* bgw,
                   const float* ballw, bool moments, double* partial_f2, void* partial_m,
                   unsigned int* counter, double* out, const double* bgm, int* overflow);
void launch_source_f64(cudaStream_t st, int grid, const double* delta, int n, Grid fh,
                       Grid fl, double S, bool moments, double* partial,
                       unsigned int* counter, double* out);
cudaError_t launch_ade_sweep(cudaStream_t st, Grid ph, Grid pl, Grid fh, Grid fl,
                             double fscale, int periodic, double lam, bool upward);
void launch_diff_rhs(cudaStream_t st, int grid, Grid sh, Grid sl, double scale, Grid ph,
                     Grid pl, double sig, Grid gh, Grid gl, Grid qh, Grid ql, bool stash,
                     double* partial, unsigned int* counter, double* out);
// Dirichlet ghost values of the open boundary into (ph, pl), and into
// (*ph2, *pl2) as well when they are given
// The ball solve's boundary values (multipoles mom, source factor S) at the
// cells of the padded cube outside the mask of ph (its mask fields), in both
// potential buffers.
void launch_ball_ghosts(cudaStream_t st, Grid ph, Grid pl, Grid ph2, Grid pl2, int n, int lo,
                        const double* mom, double S);
void launch_boundary(cudaStream_t st, Grid ph, Grid pl, int n, int lo, const double* mom,
                     double S, bool want_lo, const Grid* ph2 = nullptr,
                     const Grid* pl2 = nullptr);

// k_mg.cu
// d0: base diagonal of the operator sum_nb u - d0 u (6: Poisson; 6 + sig h^2:
// an implicit diffusion substep)
// zero_start: 0, or 1 for a first red sweep from a zero iterate, 2 for the
// black sweep right after it (its cells' own values are taken as zero)
void launch_rbgs(cudaStream_t st, Grid u, Grid b, float h2, int color, int periodic,
                 float gam, int zero_start = 0, float d0 = 6.0f);
// The rest of a V-cycle from the first level of side <= cmg_top_side(
// cmg_cluster()) in one thread-block cluster (k_cmg.cu): cmg_prepare picks
// the largest cluster the GPU holds (16 CTAs: levels <= 64^3; 8: <= 32^3;
// one CTA: <= 16^3), outside any stream capture.
cudaError_t cmg_prepare();
int cmg_cluster();
int cmg_top_side(int cl);
// dynamic shared memory of a coarse-level launch from tops up to `top`, and
// whether one-CTA tops <= 16 take the constant-side form (cmg_fast.cuh; 0
// with PM_CMG_GENERIC set: the generic form, the same bits)
int cmg_smem_bytes(int top);
int cmg_fast();
void launch_cmg(cudaStream_t st, Grid u, Grid b, int level, int periodic, int sweeps,
                bool zero_top, float sig0);
void launch_resid_restrict(cudaStream_t st, Grid u, Grid b, float inv_h2, Grid uc, Grid bc,
                           int periodic, float gam, float d0 = 6.0f);
void launch_prolong_to(cudaStream_t st, Grid uc, Grid u, Grid w, int periodic, float gam_c);
void launch_copy_ghosts(cudaStream_t st, Grid src, Grid d1, Grid d2);
// the fused two-sweep smoother (k_rbgs2.cu): tile height ty 16, 24 or 32
// (the ball solve's masked grids: 16), zc planes per CTA (0: by rbgs2_zchunk)
void launch_rbgs2(cudaStream_t st, Grid win, Grid wout, Grid b, float h2, int periodic, float gam,
                  bool zero_start, int zc = 0, float d0 = 6.0f, int ty = 16);
int rbgs2_zchunk(int s, int ty = 16);
bool rbgs2_tile_ok(int ty);
cudaError_t mg_prepare();
void launch_prolong(cudaStream_t st, Grid uc, Grid u, int periodic, float gam_c);
// residual of Phi (e == NULL) or of Phi + e written to (qh, ql) (e != NULL)
void launch_defect(cudaStream_t st, Grid ph, Grid pl, const Grid* e, Grid qh, Grid ql,
                   Grid fh, Grid fl, Grid rb, int periodic, bool write_r, double* partial,
                   unsigned int* counter, double* out, double d0 = 6.0);
int defect_blocks(int s);
void launch_correct(cudaStream_t st, Grid ph, Grid pl, Grid e);
void launch_to_dense(cudaStream_t st, Grid g, float* d, bool add);
void launch_from_dense(cudaStream_t st, const float* d, Grid g, bool add);
void launch_predict(cudaStream_t st, Grid ph, Grid pl, Grid qh, Grid ql, float w, bool pair);
void launch_fill(cudaStream_t st, Grid g, float v, bool with_ghost);
void launch_phi_out(cudaStream_t st, Grid ph, Grid pl, float* out32, double* out64,
                    double shift);
void launch_sum_phi(cudaStream_t st, Grid ph, Grid pl, double* partial, unsigned int* counter,
                    double* out);

// k_part.cu
constexpr int BALL_GL = 16;  // Gauss-Legendre points per axis and quadrant
struct BallRule {
  float xi[BALL_GL];  // nodes on [0, 1]
  float om[BALL_GL];  // weights on [0, 1] times the tent 1 - xi
};
void launch_ball_w(cudaStream_t st, float* W, int n, int lo, int s, double R,
                   const BallRule& rule, double* partial, unsigned int* counter, double* out);
void launch_drift_deposit_tsc(cudaStream_t st, long long N, float4* pos, const float4* mom,
                              float c0, bool drift, int n, int lo, int s, int periodic,
                              unsigned long long* rho, unsigned long long* escaped);
void launch_gather_tsc(cudaStream_t st, float4* pos, float4* mom, long long N,
                       const float4* G, int n, int lo, int s, int periodic, float kick,
                       float c2, int do_flag, float klo, float khi, unsigned char* flags,
                       unsigned int* block_keep, float4* forces,
                       unsigned long long* escaped);
// Particles per block of the particle kernels (gather, keep flags, block
// scan, stable scatter): KT threads of KITEMS particles each.  Callers that
// size per-block scratch themselves use PART_CHUNK.
constexpr int KT = 256;
constexpr int KITEMS = 4;
constexpr int PART_CHUNK = KT * KITEMS;
// Learned guess: the forward 3x3x3 convolution as a tensor-core implicit
// GEMM read straight from a staged input block (k_conv.cu).  conv_fast_side
// gives the output block side for a layer (0: not applicable), wf the
// weights packed by launch_pack_wf ([n][conv_fast_kf(cin)] BF16);
// launch_conv_fast returns false if the kernel could not be configured.
int conv_fast_side(int cin, int cout);
int conv_fast_kf(int cin);
void launch_pack_wf(cudaStream_t st, const float* w, int cin, int cout, int n, void* wf);
bool launch_conv_fast(cudaStream_t st, const void* in, int B, int S, int per, int cin,
                      const void* wf, int n, int T, const float* bias, int cout, int relu,
                      void* out_bf, float* out_f, int* err);
int gkd_blocks(long long N);
// G: gradient field of k_grad (NULL: differences taken from Phi directly)
void launch_gather_kick_drift(cudaStream_t st, float4* pos, float4* mom, long long N,
                              const float* ph, const float* pl, const float4* G, int n, int lo,
                              int s, int periodic, float kick, float c2, bool do_flag, float klo,
                              float khi, KeepBall kb, unsigned char* flags,
                              unsigned int* block_keep, float4* forces,
                              unsigned long long* escaped);
void launch_grad(cudaStream_t st, const float* ph, const float* pl, int n, int lo, int s,
                 int periodic, float4* G);
void launch_flag(cudaStream_t st, const float4* pos, long long N, float klo, float khi,
                 unsigned char* flags, unsigned int* block_keep, KeepBall kb);
void launch_scan_blocks(cudaStream_t st, const unsigned int* cnt, unsigned long long* off,
                        int nblk, unsigned long long* n_keep);
void launch_scatter(cudaStream_t st, const float4* pos, const float4* mom, long long N,
                    const unsigned char* flags, const unsigned long long* keep_off,
                    float4* pos_out, float4* mom_out, float4* lc_pos, float4* lc_mom,
                    long long lc_base, float a_cross);
void launch_flag_record(cudaStream_t st, const float4* pos, const float4* mom, long long N,
                        float klo, float khi, unsigned char* flags, unsigned int* block_cnt,
                        KeepBall kb);
void launch_record(cudaStream_t st, const float4* pos, float4* mom, long long N,
                   const unsigned char* flags, const unsigned long long* off, float4* lc_pos,
                   float4* lc_mom, long long lc_base, long long lc_cap, float a_cross);

// k_pk.cu
void launch_pk_delta(cudaStream_t st, const unsigned long long* rho, float* delta, int n,
                     double inv_mean);
void launch_pk_bin(cudaStream_t st, const float2* dk, int n, double box, double shot,
                   int n_bins, double* acc);
void launch_pk_jing(cudaStream_t st, const float2* dk, int n, double box, double shot,
                    int n_bins, int m, const double* nu, double* acc);

}  // namespace pm

namespace pm {

// ---------------------------------------------------------------------------
// Descriptors of batched launches (one entry per member realisation r; the
// fields are the arguments of the single-realisation kernel of that name,
// plus the member's grid dimensions).
// ---------------------------------------------------------------------------
struct RbgsDesc {
  Grid u, b;
  float h2, gam;
  int color, periodic, zero_start;
  int r, gx, gy, gz;
};
struct RestrictDesc {
  Grid u, b, uc, bc;
  float inv_h2, gam;
  int periodic;
  int r, gx, gy, gz;
};
struct ProlongDesc {
  Grid uc, u;
  float gam_c;
  int periodic;
  int r, gx, gy, gz;
};
struct CmgDesc {
  Grid u, b;
  int level, periodic, sweeps, zero_top;
  int r, gx, gy, gz;
};
struct DefectDesc {
  Grid ph, pl, e, qh, ql, fh, fl, rb;
  int periodic, write_r, correct;
  double* partial;
  unsigned int* counter;
  double* out;
  // a solve decided on the device: ph/pl the buffer it started in, qh/ql the
  // other, iters[r] the V-cycles run so far; after V-cycle k >= 1 the
  // correction moves the potential from the buffer of parity k - 1 into that
  // of parity k (iters NULL: `correct` decides)
  const int* iters;
  int r, gx, gy, gz;
};
struct PredictDesc {
  Grid ph, pl, qh, ql;
  float w;
  int pair;
  int r, gx, gy, gz;
};
struct DepositDesc {
  float4* pos;
  const float4* mom;
  long long N;
  float c0;
  int n, lo, s, periodic;
  unsigned long long* rho;
  unsigned long long* escaped;
  int r, gx, gy, gz;
};
struct SourceDesc {
  unsigned long long* rho;
  int n, lo, s;
  Grid fh, fl;
  df invM, S;
  const df* bgw;
  int moments;
  double* partial_f2;
  void* partial_m;
  unsigned int* counter;
  double* out;
  const double* bgm;
  double invM_d;
  int* overflow;
  int r, gx, gy, gz;
};
struct BoundaryDesc {
  Grid ph, pl;
  int n, lo;
  const double* mom;
  double S;
  int want_lo;
  int r, gx, gy, gz;
};
// the gradient field of a realisation's potential (ph, pl: the padded mesh;
// the persistent solve takes (ph_alt, pl_alt) instead when the V-cycles it
// ran are odd in number)
struct GradDesc {
  const float *ph, *pl, *ph_alt, *pl_alt;
  const int* flip;  // the graph solve: (ph_alt, pl_alt) where flip[r] is odd
  int n, lo, s, periodic;
  float4* G;
  int r, gx, gy, gz;
};
struct GatherDesc {
  float4 *pos, *mom;
  long long N;
  const float4* G;  // the gradient field, (n + 2)^3
  int n, lo, s, periodic;
  float kick, c2;
  int do_flag;
  float klo, khi;
  unsigned char* flags;
  unsigned int* block_keep;
  float4* forces;
  unsigned long long* escaped;
  int r, gx, gy, gz;
};
struct ScanDesc {
  const unsigned int* cnt;
  unsigned long long* off;
  int nblk;
  unsigned long long* n_keep;
  int r, gx, gy, gz;
};
struct ScatterDesc {
  const float4 *pos, *mom;
  long long N;
  const unsigned char* flags;
  const unsigned long long* keep_off;
  float4 *pos_out, *mom_out, *lc_pos, *lc_mom;
  long long lc_base;
  float a_cross;
  int r, gx, gy, gz;
};

// batched launchers: `grid` blocks (the members' total, or more), tables in
// device memory, `active` (may be NULL) masks realisations by index
void launch_rbgs_b(cudaStream_t st, int grid, const RbgsDesc* d, const BTable* t,
                   const int* active, int bx, int by);
void launch_restrict_b(cudaStream_t st, int grid, const RestrictDesc* d, const BTable* t,
                       const int* active);
void launch_prolong_b(cudaStream_t st, int grid, const ProlongDesc* d, const BTable* t,
                      const int* active);
// batched: cluster c solves entry c of d (n_desc entries, one per
// realisation; entries whose realisation is inactive are skipped); shared
// memory for tops up to max_top
void launch_cmg_b(cudaStream_t st, int n_desc, int max_top, const CmgDesc* d,
                  const int* active);
// ---------------------------------------------------------------------------
// Persistent batched solve: one cooperative launch runs defect, convergence
// test and V-cycle of every realisation until all have converged (or reached
// their V-cycle limit); phases are separated by a grid-wide barrier whose
// waits end after a time limit.
// ---------------------------------------------------------------------------
// barrier state (zeroed before a launch): arrivals, generation, and the error
// (1 = a wait ran out; every later wait then ends at once) with the phase it
// ran out in
struct GridBar {
  unsigned count, gen;
  int err, where;
};
enum { SLOT_RBGS = 0, SLOT_RESTRICT = 1, SLOT_PROLONG = 2, SLOT_CMG = 3 };
struct SolveSlot {
  int kind;          // SLOT_*
  int n;             // SLOT_CMG: descriptors
  const void* d;     // RbgsDesc / RestrictDesc / ProlongDesc / CmgDesc array
  const BTable* t;   // block table (unused for SLOT_CMG)
};
struct SolveArgs {
  const GradDesc* grad;   // per realisation: the gradient field of the final potential,
  const BTable* grad_t;   // written once every realisation has converged
  const DefectDesc* def;  // per realisation: the buffer it starts in (ph, pl), the other
  const BTable* def_t;    // one (qh, ql); defect after V-cycle it applies e into
  const SolveSlot* slots; // buffer it & 1 (relative to the start) from the other
  int n_slots;            // the V-cycle, in launch order
  int R;
  const double* scal;     // 16 per realisation: [0] ||f||^2, [11] ||r||^2 (written here)
  const double* rtol;     // R each
  const int* maxv;
  int* iters;             // out: V-cycles run
  int* failed;            // out: 1 where max_vcycles was reached first
  double* rel;            // out: the last relative residual
  GridBar* bar;
  unsigned long long limit_ns;  // longest wait at one barrier
  int extra;              // arrivals a barrier waits for beyond the grid (0; > 0 only to
                          // test the time limit: no barrier then completes)
  int fast_coarse;        // cmg_fast()
};
// The graph form of a device-decided batched solve: kb_solve_init marks the
// R realisations active with no V-cycles run; kb_converged (after each
// batched defect) takes each active realisation's decision as a single
// context's host loop does (stop at ||r|| / ||f|| <= rtol or f = 0, fail at
// max_vcycles, else count the next V-cycle) and sets the conditional handle
// of the graph's while loop to whether any realisation is still active.
void launch_solve_init_b(cudaStream_t st, int R, int* active, int* iters, int* failed);
void launch_converged_b(cudaStream_t st, int R, const double* scal, const double* rtol,
                        const int* maxv, int* active, int* iters, int* failed, double* rel,
                        cudaGraphConditionalHandle loop);
// blocks of one persistent solve launch (all co-resident), and its launch
int solve_grid_b();
cudaError_t launch_solve_b(cudaStream_t st, const SolveArgs& a);
void launch_defect_b(cudaStream_t st, int grid, const DefectDesc* d, const BTable* t,
                     const int* active);
void launch_predict_b(cudaStream_t st, int grid, const PredictDesc* d, const BTable* t);
void launch_deposit_b(cudaStream_t st, int grid, const DepositDesc* d, const BTable* t);
void launch_source_b(cudaStream_t st, int grid, const SourceDesc* d, const BTable* t);
void launch_boundary_b(cudaStream_t st, int grid, const BoundaryDesc* d, const BTable* t);
void launch_grad_b(cudaStream_t st, int grid, const GradDesc* d, const BTable* t);
void launch_gather_b(cudaStream_t st, int grid, const GatherDesc* d, const BTable* t);
void launch_scan_b(cudaStream_t st, int grid, const ScanDesc* d, const BTable* t);
void launch_scatter_b(cudaStream_t st, int grid, const ScatterDesc* d, const BTable* t);

// grid shapes of the single-realisation launches (blocks per dimension)
dim3 rbgs_grid(int s);
dim3 rbgs_grid(int s, int bx, int by);
dim3 full_grid(int s);
dim3 defect_grid(int s);
// grids of the batched colour pass, restriction, prolongation and
// prediction tables (BZ planes per block)
dim3 rbgs_grid_b(int s, int bx, int by);
dim3 full_grid_b(int s);
dim3 source_grid(int s);
int boundary_blocks(int s);
int deposit_blocks(long long N);

}  // namespace pm

namespace pm {
// k_nn.cu
void launch_wait_selftest(cudaStream_t st, int arrive, long long limit, int* gave_up);
void launch_gemm_tc(cudaStream_t st, const void* A, const void* B, float* C, int M, int N,
                    int K, int* err);
void launch_conv_fwd(cudaStream_t st, const void* in, int B, int D, int H, int W, int per,
                     int cin, const void* wp, int n, int kp, const float* bias, int cout,
                     int relu, void* out_bf, float* out_f, int* err);
void launch_conv_wgrad(cudaStream_t st, const void* in, int B, int D, int H, int W, int per,
                       int cin, const void* dy, int cout, int n, float* dw, int* err);
void launch_resid_loss(cudaStream_t st, const float* y, const float* target, int B, int S,
                       int per, const float* tscale, float* d, float* q, void* dy, double* loss);
void launch_pack_w(cudaStream_t st, const float* w, int cin, int cout, void* wp, int n, int kp,
                   void* wt, int nt, int kpt);
void launch_relu_bwd(cudaStream_t st, void* dy, const void* y, long long n);
void launch_pool2(cudaStream_t st, const void* in, int B, int D, int H, int W, int C, void* out);
void launch_pool2_bwd(cudaStream_t st, const void* dout, int B, int D, int H, int W, int C,
                      void* din);
void launch_up2(cudaStream_t st, const void* in, int B, int D, int H, int W, int C, void* out,
                int Cout, int c0);
void launch_up2_bwd(cudaStream_t st, const void* dout, int B, int D, int H, int W, int Cout,
                    int c0, int C, void* din);
void launch_chan_copy(cudaStream_t st, const void* src, long long nvox, int C, int Csrc, int s0,
                      void* dst, int Cdst, int c0, bool add);
void launch_nn_input(cudaStream_t st, const float* f, long long vps, const float* scale, int B,
                     void* x);
void launch_mse(cudaStream_t st, const float* y, const float* target, long long vps,
                const float* tscale, int B, void* dy, double* loss);
void launch_bias_grad(cudaStream_t st, const void* dy, long long nvox, int cout, int coutp,
                      float* db);
void launch_adam(cudaStream_t st, float* w, const float* g, float* m, float* v, long long n,
                 float lr, float b1, float b2, float eps, float c1, float c2);
void launch_nn_output(cudaStream_t st, const float* y, long long vps, const float* scale, int B,
                      float* phi);
// the learned guess as seen by the solver (nn_net.cu)
bool guess_fits(const pm_guess* g, int S);
pm_status guess_apply(pm_guess* g, cudaStream_t st, const float* src, int S, int per, float* out);
pm_status guess_check(pm_guess* g, cudaStream_t st);
}  // namespace pm
