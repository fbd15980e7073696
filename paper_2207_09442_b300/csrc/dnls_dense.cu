// Batched dense SPD solves through the tensor-core factor and FP64 conjugate gradients of
// dnls_tc.cuh (the dense solve of Sec. 2's normal equations, as the reduced camera systems of
// Sec. 4.2 use it), exposed on their own so that the factor can be checked against plain dense
// linear algebra.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "../../include/dnls.h"
#include "dnls_tc.cuh"

namespace {

using dnls::tc::Region;

// A_ij of problem b from the caller's row-major [batch, n, n] array
struct DenseSrc {
  const double* A;
  int nn;
  __device__ int n(int) const { return nn; }
  __device__ double val(int b, int i, int j) const { return A[((int64_t)b * nn + i) * nn + j]; }
};

struct DenseIO {
  const double* rhs;
  double* x;
  int32_t* steps;
  double* resid;
  int nn;
  __device__ int n(int) const { return nn; }
  __device__ double rhs_of(int b, int i) const { return rhs[(int64_t)b * nn + i]; }
  __device__ void out(int b, int i, double v) const { x[(int64_t)b * nn + i] = v; }
  __device__ void report(int b, int st, double res, bool ok) const {
    if (steps) steps[b] = ok ? st : -2;
    if (resid) resid[b] = res;
  }
  __device__ void factor_failed(int b, int fstat) const {
    if (steps) steps[b] = fstat == 2 ? -3 : -1;
  }
};

int padded(int n) { return ((n + dnls::tc::kSlab - 1) / dnls::tc::kSlab) * dnls::tc::kSlab; }

// per-problem offsets (int64) and orders (int32) ahead of the regions
int64_t table_bytes(int B) { return dnls::tc::a256((int64_t)B * 12 + 64); }

__global__ void k_dense_init(int B, int n, int np, int64_t region_bytes, int64_t first, int64_t* off,
                             int32_t* npv, char* base, double* x, int32_t* steps, double* resid) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < B) {
    off[t] = first + t * region_bytes;
    npv[t] = np;
    dnls::tc::Hdr* h = (dnls::tc::Hdr*)(base + first + t * region_bytes);
    h->fstat = 1;  // until the factor launch has run
    if (steps) steps[t] = -1;
    if (resid) resid[t] = __longlong_as_double(0x7ff8000000000000ll);
  }
  if (t < (int64_t)B * n) x[t] = __longlong_as_double(0x7ff8000000000000ll);
}

// cluster size for the solve: enough CTAs per problem to cover the SMs, at least 32 rows each
int pick_cluster(int B, int np, int steps, int sms) {
  if (steps <= 0) return 1;
  int kc = 1;
  while (kc < dnls::tc::kMaxCluster && (int64_t)B * kc * 2 <= sms && np / (kc * 2) >= 32) kc *= 2;
  return kc;
}

}  // namespace


extern "C" {

dnls_status dnls_dense_spd_workspace_size(int32_t batch, int32_t n, size_t* bytes) {
  if (!bytes || batch < 1 || n < 1) return DNLS_ERR_ARG;
  if (n > DNLS_DENSE_MAX_N) return DNLS_ERR_UNSUPPORTED;
  *bytes = (size_t)(table_bytes(batch) + (int64_t)batch * Region::of(padded(n)).bytes);
  return DNLS_OK;
}

dnls_status dnls_dense_spd_solve(int32_t batch, int32_t n, const double* A, const double* rhs, double* x,
                                 int32_t max_steps, double tol, void* workspace, size_t workspace_bytes,
                                 void* stream, int32_t* steps, double* resid) {
  if (batch < 1 || n < 1 || !A || !rhs || !x || max_steps < 0 || !(tol >= 0.0)) return DNLS_ERR_ARG;
  if (n > DNLS_DENSE_MAX_N) return DNLS_ERR_UNSUPPORTED;
  size_t need = 0;
  dnls_dense_spd_workspace_size(batch, n, &need);
  if (!workspace || ((uintptr_t)workspace & 255) || workspace_bytes < need) return DNLS_ERR_WORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return DNLS_ERR_CUDA;
  const int np = padded(n);
  const int64_t rbytes = Region::of(np).bytes, first = table_bytes(batch);
  char* base = (char*)workspace;
  int64_t* off = (int64_t*)base;
  int32_t* npv = (int32_t*)(base + (int64_t)batch * 8);
  const int64_t work = std::max<int64_t>(batch, (int64_t)batch * n);
  k_dense_init<<<(unsigned)((work + 255) / 256), 256, 0, st>>>(batch, n, np, rbytes, first, off, npv, base, x, steps,
                                                               resid);
  dnls::tc::Batch tb = {batch, np, base, off, npv, nullptr, nullptr, nullptr, 0};
  DenseSrc src = {A, n};
  dnls::tc::k_tc_densify<DenseSrc><<<dim3(np / dnls::tc::kNb, batch), 256, 0, st>>>(tb, src);
  if (dnls::tc::launch_factor(tb, st) != cudaSuccess || dnls::tc::launch_inverse(tb, st) != cudaSuccess)
    return DNLS_ERR_CUDA;
  DenseIO io = {rhs, x, steps, resid, n};
  const int kc = pick_cluster(batch, np, max_steps, sms);
  if (dnls::tc::launch_pcg(tb, io, max_steps, tol, kc, st) != cudaSuccess) return DNLS_ERR_CUDA;
  return cudaGetLastError() == cudaSuccess ? DNLS_OK : DNLS_ERR_CUDA;
}

}  // extern "C"
