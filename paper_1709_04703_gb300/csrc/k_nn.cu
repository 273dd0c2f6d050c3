// Learned initial guess: BF16 tensor-core (tcgen05, TMEM accumulator)
// kernels of a small 3-D convolutional network and its training.
//
//   * k_gemm_tc      plain C = A B^T (validation of the tile engine)
//   * k_conv_fwd     implicit-GEMM 3x3x3 "same" convolution, channels-last
//                    activations; M = 128 voxels, N = output channels,
//                    K = 27 * input channels (im2col gathered into shared
//                    memory), FP32 accumulation, bias + optional ReLU,
//                    BF16 and/or FP32 output
//   * k_conv_wgrad   weight gradient dW = sum_v in(v + tap) dY(v): M = 27 * Cin
//                    rows, N = Cout, K = voxels split across blocks
//   * elementwise    ReLU backward, 2x average pooling / nearest upsampling
//                    (and their backward), channel concatenation, MSE, Adam
// The input-gradient of a convolution is the forward convolution of the
// output-gradient with mirrored, transposed weights (k_conv_wt_flip).
#include <cuda_bf16.h>

#include "pm_kernels.cuh"
#include "tc_gemm.cuh"

namespace pm {

using bf16 = __nv_bfloat16;
constexpr long long TC_WAIT_LIMIT = 20000000;  // mbarrier polls before giving up

// ---------------------------------------------------------------------------
// Shared tile loop.  FillA(kt, sA) / FillB(kt, sB) stage K-chunk kt (KC wide)
// of A (128 rows) and B (N rows) into shared memory in the canonical layout;
// the loop issues KC/16 MMAs per chunk from one thread and waits on the
// mbarrier before the next chunk reuses the buffers.  Returns false on a
// timed-out wait (the error word is set; the caller still frees TMEM).
// ---------------------------------------------------------------------------
template <int N, int KC, class FillA, class FillB>
__device__ bool tc_mainloop(FillA fa, FillB fb, int ktiles, uint32_t taddr, uint8_t* sA,
                            uint8_t* sB, uint32_t mbar, uint32_t& phase, int* err) {
  constexpr uint32_t IDESC = tc::idesc_bf16(tc::TM, N);
  constexpr uint32_t SBO = KC * 16;
  bool ok = true;
  for (int kt = 0; kt < ktiles; ++kt) {
    fa(kt, sA);
    fb(kt, sB);
    tc::fence_async_smem();
    __syncthreads();
    tc::tc_fence_after();
    if (threadIdx.x == 0) {
      const uint32_t a0 = tc::smem_u32(sA), b0 = tc::smem_u32(sB);
#pragma unroll
      for (int s = 0; s < KC / 16; ++s) {
        uint64_t ad = tc::smem_desc(a0 + 256u * s, 128u, SBO);
        uint64_t bd = tc::smem_desc(b0 + 256u * s, 128u, SBO);
        tc::mma_bf16(taddr, ad, bd, IDESC, (kt > 0 || s > 0) ? 1u : 0u);
      }
      tc::mma_commit(mbar);
    }
    bool done = tc::mbar_wait(mbar, phase, TC_WAIT_LIMIT);
    phase ^= 1u;
    if (!done) {
      if (threadIdx.x == 0) atomicOr(err, 1);
      ok = false;
      // give the MMAs one more bounded wait before the buffers are left
      tc::mbar_wait(mbar, phase ^ 1u, TC_WAIT_LIMIT);
      break;
    }
    tc::tc_fence_after();
    __syncthreads();
  }
  return ok;
}

// Shared setup/teardown around a tile: TMEM allocation by warp 0, mbarrier.
struct TcCtx {
  uint32_t taddr;
  uint32_t mbar;
};

template <int NCOLS>
__device__ __forceinline__ TcCtx tc_begin(uint32_t* tslot, uint64_t* mbar_slot) {
  if (threadIdx.x < 32) tc::tmem_alloc(tslot, NCOLS);
  if (threadIdx.x == 0) tc::mbar_init(tc::smem_u32(mbar_slot), 1);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  return TcCtx{*tslot, tc::smem_u32(mbar_slot)};
}

template <int NCOLS>
__device__ __forceinline__ void tc_end(const TcCtx& c) {
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (threadIdx.x < 32) tc::tmem_free(c.taddr, NCOLS);
}

// Copy rows x (KC/8) 16-byte vectors into the canonical tile; vec(r, v)
// returns the 8 bf16 of row r, K columns [8v, 8v + 8) as a uint4.
template <int KC, class Vec>
__device__ __forceinline__ void fill_tile(uint8_t* s, int rows, Vec vec) {
  constexpr int VPR = KC / 8;
  for (int idx = threadIdx.x; idx < rows * VPR; idx += blockDim.x) {
    int r = idx / VPR, v = idx - r * VPR;
    *reinterpret_cast<uint4*>(s + tc::tile_offset(r, 8 * v, KC)) = vec(r, v);
  }
}

// ---------------------------------------------------------------------------
// Plain GEMM C[M x N] = A[M x K] B[N x K]^T (row-major bf16 inputs, FP32 C).
// M % 128 == 0, K % 64 == 0.
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(128) k_gemm_tc(const bf16* __restrict__ A,
                                                 const bf16* __restrict__ B,
                                                 float* __restrict__ C, int M, int K,
                                                 int* err) {
  constexpr int KC = 64;
  __shared__ __align__(1024) uint8_t sA[tc::TM * KC * 2];
  __shared__ __align__(1024) uint8_t sB[N * KC * 2];
  __shared__ uint32_t tslot;
  __shared__ __align__(8) uint64_t mbar;
  constexpr int NC = tc::tmem_cols(N);
  TcCtx c = tc_begin<NC>(&tslot, &mbar);
  const int m0 = blockIdx.x * tc::TM;
  uint32_t phase = 0;
  auto fa = [&](int kt, uint8_t* s) {
    fill_tile<KC>(s, tc::TM, [&](int r, int v) {
      return *reinterpret_cast<const uint4*>(A + (long long)(m0 + r) * K + kt * KC + 8 * v);
    });
  };
  auto fb = [&](int kt, uint8_t* s) {
    fill_tile<KC>(s, N, [&](int r, int v) {
      return *reinterpret_cast<const uint4*>(B + (long long)r * K + kt * KC + 8 * v);
    });
  };
  bool ok = tc_mainloop<N, KC>(fa, fb, K / KC, c.taddr, sA, sB, c.mbar, phase, err);
  if (ok) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = m0 + 32 * w + lane;
#pragma unroll
    for (int col = 0; col < N; col += 8) {
      float v[8];
      tc::tmem_ld8(c.taddr, w, col, v);
#pragma unroll
      for (int q = 0; q < 8; ++q) C[(long long)row * N + col + q] = v[q];
    }
  }
  tc_end<NC>(c);
}

void launch_gemm_tc(cudaStream_t st, const void* A, const void* B, float* C, int M, int N,
                    int K, int* err) {
  dim3 grid(M / tc::TM);
  switch (N) {
    case 16: k_gemm_tc<16><<<grid, 128, 0, st>>>((const bf16*)A, (const bf16*)B, C, M, K, err); break;
    case 32: k_gemm_tc<32><<<grid, 128, 0, st>>>((const bf16*)A, (const bf16*)B, C, M, K, err); break;
    case 64: k_gemm_tc<64><<<grid, 128, 0, st>>>((const bf16*)A, (const bf16*)B, C, M, K, err); break;
    case 128: k_gemm_tc<128><<<grid, 128, 0, st>>>((const bf16*)A, (const bf16*)B, C, M, K, err); break;
    default: return;
  }
  note_launch();
}

}  // namespace pm
