// The tensor-core Cholesky factor of dnls_tc.cuh: one CTA per problem, the 128-row slab being
// factored held in tensor memory, trailing updates as tcgen05.mma on BF16-split panels.
#include "dnls_tc.cuh"

namespace dnls {
namespace tc {
namespace {

// bf16 round-to-nearest of x and the FP32 remainder (exact: x - bf16(x) is representable)
__device__ __forceinline__ uint32_t bf16_bits(float x) {
  return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x));
}
__device__ __forceinline__ float bf16_val(uint32_t h) {
  return __uint_as_float(h << 16);
}

// One CTA of kFactorThreads per problem; shared memory kFactorSmem; one CTA per SM (the
// shared memory ensures it), so the tensor-memory allocation never waits for another CTA.
// Attempts shifts sigma = 0, 1e-5, 1e-3 (of the unit-scale diagonal) until every pivot is
// positive.  limit_ns bounds every wait on an mbarrier.
__global__ void __launch_bounds__(kFactorThreads, 1) k_tc_factor(Batch tb, uint64_t limit_ns) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int b = blockIdx.x;
  if (b >= tb.B || !tb.on(b)) return;
  const int np = tb.np[b];
  const int S = np / kSlab, P = np / kNb;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  char* R = tb.base + tb.off[b];
  Hdr* hdr = (Hdr*)R;
  const Region rg = Region::of(np);
  const double* A = (const double*)(R + rg.A);
  float* Lg = (float*)(R + rg.L);
  float* Linv_g = (float*)(R + rg.Linv);
  unsigned char* split_g = (unsigned char*)(R + rg.split);

  unsigned char* bufs = sm;
  float* Linv_s = (float*)(sm + 2 * kBufBytes);
  float* Ls = Linv_s + kMaxPanels * 1024;
  float* rdiag = Ls + 32 * 33;
  uint64_t* bars = (uint64_t*)(rdiag + 32);  // [0] MMA done, [1], [2] bulk copies into buffer 0 / 1
  uint32_t* tslot = (uint32_t*)(bars + 3);
  int* sflag = (int*)(tslot + 1);  // [0] error (2 = timeout), [1] failed pivot

  const uint32_t ncols = np <= 128 ? 128u : (np <= 256 ? 256u : 512u);
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    mbar_init(&bars[2], 1);
    mbar_fence_init();
    sflag[0] = 0;
  }
  if (warp == 0) tmem_alloc(tslot, ncols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t tlane = tmem + ((uint32_t)(warp * 32) << 16);  // this warp's lane quarter
  uint32_t mma_phase = 0, tma_phase[2] = {0, 0};
  bool mma_pending = false;
  int result = 1;
  double shift = 0.0;
  int attempt = 0;
  for (; attempt < 3 && result == 1; ++attempt) {
    shift = attempt == 0 ? 0.0 : (attempt == 1 ? 1e-5 : 1e-3);
    if (tid == 0) sflag[1] = 0;
    __syncthreads();
    bool failed = false;
    for (int s = 0; s < S && !failed; ++s) {
      const int row = kSlab * s + tid;
      const int ncol_s = kSlab * (s + 1);
      // this slab's rows of A~ (lower part, shifted diagonal) into tensor memory as FP32
      for (int c0 = 0; c0 < ncol_s; c0 += 32) {
        float v[32];
        const double* Ar = A + (int64_t)row * np + c0;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int col = c0 + j;
          v[j] = col < row ? (float)Ar[j] : (col == row ? (float)(Ar[j] + shift) : 0.0f);
        }
        tmem_st32(tlane + c0, v);
      }
      for (int k = 0; k < 4 * s + 4; ++k) {
        const int buf = k & 1, kd = k - 4 * s;
        unsigned char* Bf = bufs + buf * kBufBytes;
        const int r0 = kNb * (k + 1), r1 = kSlab * s;  // rows of earlier slabs for this panel's B
        const bool has_copy = r0 < r1;
        if (mma_pending) {
          if (!mbar_wait(&bars[0], mma_phase, limit_ns)) sflag[0] = 2;
          mma_phase ^= 1;
          mma_pending = false;
        }
        tc_fence_after();
        if (tid == 0 && has_copy) {
          const uint32_t per_term = (uint32_t)(r1 - r0) * 64;
          mbar_arrive_expect_tx(&bars[1 + buf], 3 * per_term);
#pragma unroll
          for (int t = 0; t < 3; ++t)
            bulk_g2s(Bf + t * kTermBytes + (r0 / 8) * 512,
                     split_g + ((int64_t)(k * 3 + t) * (np / 8) + r0 / 8) * 512, per_term, &bars[1 + buf]);
        }
        float a[32];
        tmem_ld32(tlane + kNb * k, a);
        if (kd >= 0 && warp == kd) {
          // diagonal block: lane l holds row 32k + l; Cholesky by columns with shuffles
          bool ok = true;
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const float ajj = __shfl_sync(0xffffffffu, a[j], j);
            ok = ok && ajj > 0.0f;
            const float rs = rsqrtf(ajj);
            const float lij = lane > j ? a[j] * rs : (lane == j ? ajj * rs : 0.0f);
            a[j] = lij;
#pragma unroll
            for (int m = j + 1; m < 32; ++m) a[m] = fmaf(-lij, __shfl_sync(0xffffffffu, lij, m), a[m]);
          }
#pragma unroll
          for (int m = 0; m < 32; ++m) Ls[lane * 33 + m] = a[m];
          rdiag[lane] = 1.0f / a[lane];
          __syncwarp();
          // column `lane` of L_kk^-1 by forward substitution
          float x[32];
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            float acc = 0.0f;
#pragma unroll
            for (int m = 0; m < i; ++m) acc = fmaf(Ls[i * 33 + m], x[m], acc);
            x[i] = i < lane ? 0.0f : (i == lane ? rdiag[i] : -acc * rdiag[i]);
          }
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            Linv_s[k * 1024 + i * 32 + lane] = x[i];
            Linv_g[(int64_t)k * 1024 + i * 32 + lane] = x[i];
          }
          if (!ok && lane == 0) sflag[1] = 1;
        }
        __syncthreads();
        if (sflag[0] || sflag[1]) {
          // no MMA of this step was issued; take the bulk copy's completion before leaving
          if (tid == 0 && has_copy && !mbar_wait(&bars[1 + buf], tma_phase[buf], limit_ns)) sflag[0] = 2;
          if (has_copy) tma_phase[buf] ^= 1;
          failed = true;
          break;
        }
        // this row's entries of panel k
        float l[32];
        if (row >= kNb * k + kNb) {
          const float* Li = Linv_s + k * 1024;
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            float acc = 0.0f;
#pragma unroll
            for (int m = 0; m <= j; ++m) acc = fmaf(a[m], Li[j * 32 + m], acc);
            l[j] = acc;
          }
        } else if (row >= kNb * k) {
#pragma unroll
          for (int m = 0; m < 32; ++m) l[m] = Ls[(row - kNb * k) * 33 + m];
        } else {
#pragma unroll
          for (int m = 0; m < 32; ++m) l[m] = 0.0f;
        }
        if (row >= kNb * k) {
          float4* dst = (float4*)(Lg + (int64_t)row * np + kNb * k);
#pragma unroll
          for (int q = 0; q < 8; ++q) dst[q] = make_float4(l[4 * q], l[4 * q + 1], l[4 * q + 2], l[4 * q + 3]);
        }
        // three-term BF16 split into the shared panel buffer (MMA operands) and the global
        // staging area (B operands of later slabs)
        {
          const int64_t go = (int64_t)(row / 8) * 512 + (row % 8) * 16;
          unsigned char* gpan = split_g + (int64_t)(k * 3) * (np / 8) * 512 + go;
#pragma unroll
          for (int q = 0; q < 4; ++q) {  // K chunk q: columns 8q .. 8q+7
            uint32_t w[3][4];
#pragma unroll
            for (int e = 0; e < 8; e += 2) {
              uint32_t hp[3][2];
#pragma unroll
              for (int u = 0; u < 2; ++u) {
                const float x = l[8 * q + e + u];
                const uint32_t h0 = bf16_bits(x);
                const float e1 = x - bf16_val(h0);
                const uint32_t h1 = bf16_bits(e1);
                hp[0][u] = h0;
                hp[1][u] = h1;
                hp[2][u] = bf16_bits(e1 - bf16_val(h1));
              }
#pragma unroll
              for (int t = 0; t < 3; ++t) w[t][e / 2] = hp[t][0] | (hp[t][1] << 16);
            }
#pragma unroll
            for (int t = 0; t < 3; ++t) {
              const uint4 v4 = make_uint4(w[t][0], w[t][1], w[t][2], w[t][3]);
              *(uint4*)(Bf + t * kTermBytes + go + q * 128) = v4;
              if (s + 1 < S) *(uint4*)(gpan + (int64_t)t * (np / 8) * 512 + q * 128) = v4;
            }
          }
        }
        fence_proxy_async_smem();
        tc_fence_before();
        __syncthreads();
        const int c0 = kNb * (k + 1), c1 = ncol_s;
        if (c0 < c1) {
          if (tid == 0) {
            if (has_copy && !mbar_wait(&bars[1 + buf], tma_phase[buf], limit_ns)) sflag[0] = 2;
            tc_fence_after();
            const uint32_t abase = smem_u32(Bf) + (uint32_t)(kSlab * s / 8) * 512;
            for (int cs = c0; cs < c1; cs += 256) {
              const int N = c1 - cs < 256 ? c1 - cs : 256;
              const uint32_t id = idesc_bf16_negA(N);
              const uint32_t bbase = smem_u32(Bf) + (uint32_t)(cs / 8) * 512;
              // (A term, B term): x0y0, x0y1, x1y0, x0y2, x1y1, x2y0
              const int pa[6] = {0, 0, 1, 0, 1, 2}, pb[6] = {0, 1, 0, 2, 1, 0};
#pragma unroll
              for (int pr = 0; pr < 6; ++pr)
#pragma unroll
                for (int kk = 0; kk < 2; ++kk)
                  mma_bf16(tmem + (uint32_t)cs, sdesc(abase + pa[pr] * kTermBytes + kk * 256, 128, 512),
                           sdesc(bbase + pb[pr] * kTermBytes + kk * 256, 128, 512), id);
            }
            mma_commit(&bars[0]);
          }
          if (has_copy) tma_phase[buf] ^= 1;
          mma_pending = true;
        }
      }
    }
    __syncthreads();
    if (sflag[0]) {
      result = 2;
    } else if (!failed) {
      result = 0;
    }
  }
  if (mma_pending) {  // only after a timeout: bounded wait for the last MMA before freeing
    mbar_wait(&bars[0], mma_phase, limit_ns);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, ncols);
  if (tid == 0) {
    hdr->fstat = result;
    hdr->attempts = attempt;
    hdr->shift = shift;
    const int64_t o = (int64_t)b * tb.stride;
    if (tb.ok) tb.ok[o] = result == 0 ? 1 : 0;
    if (tb.bad && result != 0) tb.bad[o] = 1;
  }
  (void)P;
}

}  // namespace

cudaError_t launch_factor(const Batch& tb, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(k_tc_factor, cudaFuncAttributeMaxDynamicSharedMemorySize, kFactorSmem);
  if (e != cudaSuccess) return e;
  k_tc_factor<<<tb.B, kFactorThreads, kFactorSmem, st>>>(tb, 1000000000ull);
  return cudaGetLastError();
}

}  // namespace tc
}  // namespace dnls
