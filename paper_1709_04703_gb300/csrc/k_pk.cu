// Power spectrum of a particle set (Sec. 2.4: power-spectrum calculator with
// a discreteness correction; first-order form: CIC window deconvolution and
// shot-noise subtraction).  The FFT is cuFFT (a library call, off the step's
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

}  // namespace pm
