// The coarse levels of the multigrid V-cycle (Sec. 2.1, Eq. 3 on levels of
// side <= 64) resident in the distributed shared memory of one thread-block
// cluster: the levels are split over the cluster's CTAs by z planes, each
// smoothing pass, restriction and prolongation is one phase, and phases are
// separated by the cluster's hardware barrier instead of kernel launches.
// The arithmetic is that of the per-level kernels (mg_arith.cuh), so the
// results do not depend on where a level is solved.  The bottom (side <= 4
// or odd) is solved by CTA 0 alone.
#include <cstdlib>
#include <utility>

#include "cmg_dev.cuh"
#include "cmg_fast.cuh"

namespace pm {

namespace {

template <int CL>
__global__ void __launch_bounds__(CC_NT, 1) k_cmg(Grid u, Grid b, int level, int periodic,
                                                  int sweeps, int zero_top, float sig0,
                                                  int fast) {
  pdl_wait();
  pdl_release();
  extern __shared__ float cc_sm[];
  __shared__ float red[CC_NT / 32];
  if (CL == 1 && (fast || u.mbase) && fc_supported(u.s)) {
    if (u.mbase)
      fc_vcycle<CC_NT, true>(cc_sm, red, u, b, level, periodic, sweeps, zero_top, sig0);
    else
      fc_vcycle<CC_NT, false>(cc_sm, red, u, b, level, periodic, sweeps, zero_top, sig0);
    return;
  }
  if (u.mbase) return;  // not reached: masked tops (q 2^j <= 16) are all supported
  __shared__ CcLevel lev[CC_MAXL];
  __shared__ int nlev;
  if (threadIdx.x == 0) Cc<CL>::init_levels(lev, nlev, u.s, level, periodic, sig0);
  __syncthreads();
  Cc<CL> c;
  c.sm = cc_sm;
  c.my = CL == 1 ? 0 : (int)cg::this_cluster().block_rank();
  c.periodic = periodic;
  c.sweeps = sweeps;
  c.nlev = nlev;
  c.sig0 = sig0;
  c.gu = u;
  c.gb = b;
  c.V = lev;
  c.init_pointers(lev);
  __syncthreads();
  c.run(zero_top, red);
}

// batched form: cluster c solves the coarse levels of table entry c
// (realisations whose solve has converged are skipped, by whole clusters)
template <int CL>
__global__ void __launch_bounds__(CC_NT, 1) kb_cmg(const CmgDesc* d, int n_desc,
                                                   const int* active, int fast) {
  extern __shared__ float cc_sm[];
  __shared__ float red[CC_NT / 32];
  const int q = blockIdx.x / CL;
  if (q >= n_desc) return;
  const CmgDesc& e = d[q];
  if (active && !active[e.r]) return;
  if (CL == 1 && fast && fc_supported(e.u.s)) {
    fc_vcycle<CC_NT, false>(cc_sm, red, e.u, e.b, e.level, e.periodic, e.sweeps, e.zero_top,
                            0.0f);
    return;
  }
  __shared__ CcLevel lev[CC_MAXL];
  __shared__ int nlev;
  if (threadIdx.x == 0) Cc<CL>::init_levels(lev, nlev, e.u.s, e.level, e.periodic, 0.0f);
  __syncthreads();
  Cc<CL> c;
  c.sm = cc_sm;
  c.my = CL == 1 ? 0 : (int)cg::this_cluster().block_rank();
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
}

int g_cmg_cl = 1;  // CTAs per cluster of this process's launches (set by cmg_prepare)
int g_cmg_fast = 1;  // one-CTA tops <= 16 take the constant-side form (cmg_fast.cuh)

// dynamic shared memory of a coarse-level launch from tops up to `top`
int cmg_smem(int top, int CL) {
  int f = cc_layout(top, CL).floats;
  if (CL == 1 && fc_floats(FC_MAX_TOP) > f) f = fc_floats(FC_MAX_TOP);
  return (int)sizeof(float) * f;
}

template <int CL>
cudaError_t cmg_attrs() {
  const int smem = cmg_smem(cmg_top_side(CL), CL);
  cudaError_t e = cudaFuncSetAttribute(k_cmg<CL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kb_cmg<CL>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess && CL > 8) {
    e = cudaFuncSetAttribute(k_cmg<CL>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(kb_cmg<CL>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  }
  return e;
}

// can a cluster of CL CTAs with the largest layout be resident on this GPU?
template <int CL>
bool cmg_fits() {
  if (cmg_attrs<CL>() != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(CL);
  cfg.blockDim = dim3(CC_NT);
  cfg.dynamicSmemBytes = cmg_smem(cmg_top_side(CL), CL);
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, k_cmg<CL>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return n >= 1;
}

template <int CL, class K, class... Act>
void cmg_launch(K kernel, int clusters, int top, cudaStream_t st, Act&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(CL * clusters);
  cfg.blockDim = dim3(CC_NT);
  cfg.dynamicSmemBytes = cmg_smem(top, CL);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = CL > 1 ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kernel, std::forward<Act>(args)...);
}

}  // namespace

int cmg_top_side(int cl) { return cl >= 16 ? 64 : (cl >= 8 ? 32 : 16); }

int cmg_cluster() { return g_cmg_cl; }

cudaError_t cmg_prepare() {
  // the cluster of the coarse levels: 16 CTAs (levels <= 64^3), 8 (<= 32^3)
  // or one CTA (<= 16^3) when the GPU holds it; PM_NO_CLUSTER forces one CTA
  cudaError_t e = cmg_attrs<1>();
  if (e != cudaSuccess) return e;
  g_cmg_cl = 1;
  // PM_CMG_GENERIC: the generic one-CTA form for every top (the same bits)
  g_cmg_fast = getenv("PM_CMG_GENERIC") ? 0 : 1;
  if (getenv("PM_NO_CLUSTER")) return cudaSuccess;
  // PM_CMG_CLUSTER = 8 or 16 asks for a cluster.  One CTA is the default:
  // measured on the 256^3 workload (20 steps, both phases), the coarse
  // levels took 8.7 ms with one CTA (levels <= 16^3; 32^3 and 64^3 one
  // launch per phase inside the V-cycle graph), 9.3 ms with 8 CTAs (<= 32^3)
  // and 15.2 ms with 16 (<= 64^3): a pass over a 64^3 level on 16 SMs takes
  // longer than a launch over all of them, and below that the phases are
  // latency-bound either way
  const char* cap = getenv("PM_CMG_CLUSTER");
  const int want = cap ? atoi(cap) : 1;
  if (want >= 16 && cmg_fits<16>()) g_cmg_cl = 16;
  else if (want >= 8 && cmg_fits<8>()) g_cmg_cl = 8;
  return cudaSuccess;
}

int cmg_smem_bytes(int top) { return cmg_smem(top, g_cmg_cl); }

int cmg_fast() { return g_cmg_fast; }

void launch_cmg(cudaStream_t st, Grid u, Grid b, int level, int periodic, int sweeps,
                bool zero_top, float sig0) {
  const int z = zero_top ? 1 : 0;
  // the ball solve's masked levels take the one-CTA constant-side form
  switch (u.mbase ? 1 : g_cmg_cl) {
    case 16:
      cmg_launch<16>(k_cmg<16>, 1, u.s, st, u, b, level, periodic, sweeps, z, sig0, 0);
      break;
    case 8:
      cmg_launch<8>(k_cmg<8>, 1, u.s, st, u, b, level, periodic, sweeps, z, sig0, 0);
      break;
    default:
      cmg_launch<1>(k_cmg<1>, 1, u.s, st, u, b, level, periodic, sweeps, z, sig0, g_cmg_fast);
      break;
  }
  note_launch();
}

void launch_cmg_b(cudaStream_t st, int n_desc, int max_top, const CmgDesc* d, const int* active) {
  switch (g_cmg_cl) {
    case 16: cmg_launch<16>(kb_cmg<16>, n_desc, max_top, st, d, n_desc, active, 0); break;
    case 8: cmg_launch<8>(kb_cmg<8>, n_desc, max_top, st, d, n_desc, active, 0); break;
    default:
      cmg_launch<1>(kb_cmg<1>, n_desc, max_top, st, d, n_desc, active, g_cmg_fast);
      break;
  }
  note_launch();
}

}  // namespace pm
