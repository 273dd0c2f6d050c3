// Power spectrum of a particle set (Sec. 2.4: power-spectrum calculator with
// a discreteness correction): the first-order form (CIC window deconvolution
// and shot-noise subtraction) and the full alias correction of Jing (2005)
// that the paper names.  The FFT is cuFFT (a library call, off the step's
// hot path).
#include "pm_kernels.cuh"

namespace pm {

__global__ void k_pk_delta(const unsigned long long* __restrict__ rho,
                           float* __restrict__ delta, long long total, double inv_mean) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x)
    delta[t] = (float)((double)rho[t] * inv_mean - 1.0);
}

void launch_pk_delta(cudaStream_t st, const unsigned long long* rho, float* delta, int n,
                     double inv_mean) {
  long long total = (long long)n * n * n;
  k_pk_delta<<<1216, 256, 0, st>>>(rho, delta, total, inv_mean);
  note_launch();
}

// Modes of the R2C output [kz][ky][kx], kx in 0..n/2.  acc[3*b + 0..2] +=
// (modes, sum |k|, sum P) with weight 2 for 0 < kx < n/2 (the -k partner).
__global__ void k_pk_bin(const float2* __restrict__ dk, int n, double box, double shot,
                         int n_bins, double* __restrict__ acc) {
  extern __shared__ double sacc[];
  for (int q = threadIdx.x; q < 3 * n_bins; q += blockDim.x) sacc[q] = 0.0;
  __syncthreads();
  const int nx = n / 2 + 1;
  const long long total = (long long)n * n * nx;
  const double kf = 2.0 * 3.14159265358979323846 / box;
  const double h = box / n;
  const double norm = box * box * box / ((double)n * n * n * (double)n * n * n);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int ix = (int)(t % nx);
    long long r = t / nx;
    int iy = (int)(r % n);
    int iz = (int)(r / n);
    int mx = ix, my = iy <= n / 2 ? iy : iy - n, mz = iz <= n / 2 ? iz : iz - n;
    double kx = kf * mx, ky = kf * my, kz = kf * mz;
    double kmag = sqrt(kx * kx + ky * ky + kz * kz);
    int b = (int)floor(kmag / kf + 0.5) - 1;
    if (b < 0 || b >= n_bins) continue;
    double wx = mx ? sin(kx * h * 0.5) / (kx * h * 0.5) : 1.0;
    double wy = my ? sin(ky * h * 0.5) / (ky * h * 0.5) : 1.0;
    double wz = mz ? sin(kz * h * 0.5) / (kz * h * 0.5) : 1.0;
    double W = wx * wx * wy * wy * wz * wz;
    float2 c = dk[t];
    double p = ((double)c.x * c.x + (double)c.y * c.y) * norm / (W * W) - shot;
    double w = (ix == 0 || (ix == n / 2 && (n & 1) == 0)) ? 1.0 : 2.0;
    atomicAdd(&sacc[3 * b + 0], w);
    atomicAdd(&sacc[3 * b + 1], w * kmag);
    atomicAdd(&sacc[3 * b + 2], w * p);
  }
  __syncthreads();
  for (int q = threadIdx.x; q < 3 * n_bins; q += blockDim.x)
    if (sacc[q] != 0.0) atomicAdd(&acc[q], sacc[q]);
}

void launch_pk_bin(cudaStream_t st, const float2* dk, int n, double box, double shot,
                   int n_bins, double* acc) {
  size_t smem = sizeof(double) * 3 * n_bins;
  k_pk_bin<<<608, 256, smem, st>>>(dk, n, box, shot, n_bins, acc);
  note_launch();
}

// Alias-corrected modes (Jing 2005).  Per stored mode of bin b:
//   P = (P_obs - shot C1) / C2,   C1 = prod_d [1 - (2/3) sin^2 x_d],
//   C2 = sum_{n in [-m, m]^3} prod_d sinc^4(x_d + pi n_d) (r_n / r_0)^(nu_b / 2),
// x_d = k_d h / 2, r_n = sum_d (x_d + pi n_d)^2.  The alias terms are FP32
// (factorised per axis), their sum and everything else FP64.  acc as in
// k_pk_bin.
constexpr int PK_MAX_ALIAS = 3;

template <int m>
__global__ void __launch_bounds__(256) k_pk_jing(const float2* __restrict__ dk, int n,
                                                 double box, double shot, int n_bins,
                                                 const double* __restrict__ nu,
                                                 double* __restrict__ acc) {
  extern __shared__ double sacc[];
  for (int q = threadIdx.x; q < 3 * n_bins; q += blockDim.x) sacc[q] = 0.0;
  __syncthreads();
  const int nx = n / 2 + 1;
  const long long total = (long long)n * n * nx;
  const double pi = 3.14159265358979323846;
  const double kf = 2.0 * pi / box;
  const double h = box / n;
  const double norm = box * box * box / ((double)n * n * n * (double)n * n * n);
  constexpr int na = 2 * m + 1;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(t % nx);
    const long long r = t / nx;
    const int iy = (int)(r % n);
    const int iz = (int)(r / n);
    const int mv[3] = {ix, iy <= n / 2 ? iy : iy - n, iz <= n / 2 ? iz : iz - n};
    double k2 = 0.0;
    for (int d = 0; d < 3; ++d) k2 += (kf * mv[d]) * (kf * mv[d]);
    const double kmag = sqrt(k2);
    const int b = (int)floor(kmag / kf + 0.5) - 1;
    if (b < 0 || b >= n_bins) continue;
    // per-axis alias factors f[d][j] = sinc^4(x + pi n), y2[d][j] = (x + pi n)^2
    float f[3][na], y2[3][na];
    double c1 = 1.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double x = kf * mv[d] * h * 0.5;
      const double sx = sin(x);
      const double s2 = sx * sx;
      c1 *= 1.0 - (2.0 / 3.0) * s2;
#pragma unroll
      for (int j = 0; j < na; ++j) {
        const double y = x + pi * (j - m);
        y2[d][j] = (float)(y * y);
        f[d][j] = y == 0.0 ? 1.0f : (float)((s2 * s2) / (y * y * y * y));
      }
    }
    const float r0 = y2[0][m] + y2[1][m] + y2[2][m];
    const float hnu = 0.5f * (float)nu[b];
    double c2 = 0.0;
#pragma unroll
    for (int i = 0; i < na; ++i) {
#pragma unroll
      for (int j = 0; j < na; ++j) {
        const float fxy = f[0][i] * f[1][j];
        const float rxy = y2[0][i] + y2[1][j];
        if (fxy == 0.0f) continue;
#pragma unroll
        for (int l = 0; l < na; ++l) {
          const float w = fxy * f[2][l];
          if (w == 0.0f) continue;
          c2 += (double)(w * exp2f(hnu * log2f((rxy + y2[2][l]) / r0)));
        }
      }
    }
    const float2 c = dk[t];
    const double pobs = ((double)c.x * c.x + (double)c.y * c.y) * norm;
    const double p = (pobs - shot * c1) / c2;
    const double wm = (ix == 0 || (ix == n / 2 && (n & 1) == 0)) ? 1.0 : 2.0;
    atomicAdd(&sacc[3 * b + 0], wm);
    atomicAdd(&sacc[3 * b + 1], wm * kmag);
    atomicAdd(&sacc[3 * b + 2], wm * p);
  }
  __syncthreads();
  for (int q = threadIdx.x; q < 3 * n_bins; q += blockDim.x)
    if (sacc[q] != 0.0) atomicAdd(&acc[q], sacc[q]);
}

void launch_pk_jing(cudaStream_t st, const float2* dk, int n, double box, double shot,
                    int n_bins, int m, const double* nu, double* acc) {
  size_t smem = sizeof(double) * 3 * n_bins;
  switch (m) {
    case 1: k_pk_jing<1><<<1216, 256, smem, st>>>(dk, n, box, shot, n_bins, nu, acc); break;
    case 2: k_pk_jing<2><<<1216, 256, smem, st>>>(dk, n, box, shot, n_bins, nu, acc); break;
    default: k_pk_jing<PK_MAX_ALIAS><<<1216, 256, smem, st>>>(dk, n, box, shot, n_bins, nu, acc);
  }
  note_launch();
}

}  // namespace pm
