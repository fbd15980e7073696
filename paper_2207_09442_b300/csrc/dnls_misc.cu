// Small kernels of the C ABI that are not tied to a problem handle: tangent-space projection
// and lift of gradients (App. C), the status strings and the FP64 peak probe used for the
// roofline of the factorization.
#include <cuda_runtime.h>

#include "../../include/dnls.h"
#include "dnls_lie.cuh"

namespace {

// v = d/dxi L(T Exp(xi)) at 0 from G = dL/dT.
//   SE(3): v_rho = R^T G_t, v_phi = vee(M - M^T) with M = R^T G_R  (G_R the 3x3 part).
//   SE(2): v_rho = R^T (G_x, G_y), v_psi = -s G_c + c G_s.
__global__ void k_project(int kind, int64_t n, const double* T, const double* G, double* v) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  if (kind == DNLS_SE3) {
    const double* t = T + k * 12;
    const double* g = G + k * 12;
    double M[9];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j)
        M[3 * i + j] = t[0 * 4 + i] * g[0 * 4 + j] + t[1 * 4 + i] * g[1 * 4 + j] + t[2 * 4 + i] * g[2 * 4 + j];
    double* o = v + k * 6;
    for (int i = 0; i < 3; ++i) o[i] = t[0 * 4 + i] * g[3] + t[1 * 4 + i] * g[7] + t[2 * 4 + i] * g[11];
    o[3] = M[7] - M[5];
    o[4] = M[2] - M[6];
    o[5] = M[3] - M[1];
  } else {
    const double* t = T + k * 4;
    const double* g = G + k * 4;
    const double c = t[2], s = t[3];
    double* o = v + k * 3;
    o[0] = c * g[0] + s * g[1];
    o[1] = -s * g[0] + c * g[1];
    o[2] = -s * g[2] + c * g[3];
  }
}

// Minimum-norm G in the tangent space at T with proj(G) = v:
//   SE(3): G_t = R v_rho, G_R = R [v_phi]x / 2;   SE(2): G_xy = R v_rho, (G_c, G_s) = v_psi (-s, c).
__global__ void k_lift(int kind, int64_t n, const double* T, const double* v, double* G) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  if (kind == DNLS_SE3) {
    const double* t = T + k * 12;
    const double* x = v + k * 6;
    double K[9];
    dnls::hat3(x + 3, K);
    double* o = G + k * 12;
    for (int i = 0; i < 3; ++i) {
      for (int j = 0; j < 3; ++j)
        o[4 * i + j] = 0.5 * (t[4 * i + 0] * K[j] + t[4 * i + 1] * K[3 + j] + t[4 * i + 2] * K[6 + j]);
      o[4 * i + 3] = t[4 * i + 0] * x[0] + t[4 * i + 1] * x[1] + t[4 * i + 2] * x[2];
    }
  } else {
    const double* t = T + k * 4;
    const double* x = v + k * 3;
    const double c = t[2], s = t[3];
    double* o = G + k * 4;
    o[0] = c * x[0] - s * x[1];
    o[1] = s * x[0] + c * x[1];
    o[2] = -s * x[2];
    o[3] = c * x[2];
  }
}

__global__ void k_fp64_fma(double* out, int iters, double a, double b) {
  double x[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) x[c] = (double)(threadIdx.x + c) * 1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += x[c];
  out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" {

dnls_status dnls_project_grad(int32_t kind, int64_t n, const double* theta, const double* G,
                              double* v, void* stream) {
  if ((kind != DNLS_SE2 && kind != DNLS_SE3) || n < 0) return DNLS_ERR_ARG;
  if (n == 0) return DNLS_OK;
  if (!theta || !G || !v) return DNLS_ERR_ARG;
  k_project<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(kind, n, theta, G, v);
  return cudaGetLastError() == cudaSuccess ? DNLS_OK : DNLS_ERR_CUDA;
}

dnls_status dnls_lift_grad(int32_t kind, int64_t n, const double* T, const double* v, double* G,
                           void* stream) {
  if ((kind != DNLS_SE2 && kind != DNLS_SE3) || n < 0) return DNLS_ERR_ARG;
  if (n == 0) return DNLS_OK;
  if (!T || !v || !G) return DNLS_ERR_ARG;
  k_lift<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(kind, n, T, v, G);
  return cudaGetLastError() == cudaSuccess ? DNLS_OK : DNLS_ERR_CUDA;
}

const char* dnls_status_string(dnls_status s) {
  switch (s) {
    case DNLS_OK: return "DNLS_OK";
    case DNLS_ERR_ARG: return "DNLS_ERR_ARG: invalid argument";
    case DNLS_ERR_CUDA: return "DNLS_ERR_CUDA: CUDA runtime error";
    case DNLS_ERR_WORKSPACE: return "DNLS_ERR_WORKSPACE: workspace missing, misaligned or too small";
    case DNLS_ERR_TIMEOUT: return "DNLS_ERR_TIMEOUT: bounded device wait expired";
    case DNLS_ERR_UNSUPPORTED: return "DNLS_ERR_UNSUPPORTED: option combination not implemented";
  }
  return "unknown dnls_status";
}

dnls_status dnls_probe_fp64_peak(int32_t iters, void* stream, double* flops) {
  if (!flops || iters < 1) return DNLS_ERR_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return DNLS_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return DNLS_ERR_CUDA;
  const int blocks = sms * 4, threads = 256;
  double* out = nullptr;
  if (cudaMalloc(&out, sizeof(double) * blocks * threads) != cudaSuccess) return DNLS_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_fp64_fma<<<blocks, threads, 0, st>>>(out, 16, 0.999, 1e-4);
  float best = 1e30f;
  for (int r = 0; r < 3; ++r) {
    cudaEventRecord(e0, st);
    k_fp64_fma<<<blocks, threads, 0, st>>>(out, iters, 0.999, 1e-4);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  const cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess) return DNLS_ERR_CUDA;
  *flops = 2.0 * 8.0 * (double)blocks * threads * iters / (best * 1e-3);
  return DNLS_OK;
}

}  // extern "C"
