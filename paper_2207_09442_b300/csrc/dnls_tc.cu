// The tensor-core Cholesky factor of dnls_tc.cuh: one CTA per problem, the 128-row slab being
// factored held in tensor memory, trailing updates as tcgen05.mma on BF16-split panels.
#include "dnls_tc.cuh"

namespace dnls {
namespace tc {
namespace {

// bf16 round-to-nearest of x (the FP32 remainder x - bf16(x) is exactly representable)
__device__ __forceinline__ uint32_t bf16_bits(float x) {
  return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x));
}
__device__ __forceinline__ float bf16_val(uint32_t h) {
  return __uint_as_float(h << 16);
}

// One CTA of kFactorThreads per problem; shared memory kFactorSmem; one CTA per SM (the
// shared memory ensures it), so the tensor-memory allocation never waits for another CTA.
// Thread t owns row 128 s + t of slab s (tensor-memory lane t).  Per panel k of the slab:
//   1. wait for the previous panel's MMAs; start the bulk copy of this panel's B rows from
//      earlier slabs; read the row's panel columns from tensor memory;
//   2. the warp holding the diagonal block factors it (lane = row, columns by shuffles) and
//      stores L_kk^T and its reciprocal pivots in shared memory;
//   3. rows below solve l L_kk^T = a by substitution; the row's entries go to L (global) and,
//      split into three BF16 terms, to the shared panel buffer (MMA operands) and, for later
//      slabs, to the global staging area;
//   4. one thread issues the trailing update D[slab rows, columns > panel] -= A B^T as 12 MMAs
//      per 256-column chunk (6 split products x 2 K steps) and commits to an mbarrier.
// After the last panel the diagonal blocks are inverted (warp w: panels w, w+4, ...) for the
// triangular solves.  Shifts sigma = 0, 1e-5, 1e-3 (of the unit-scale diagonal) are tried until
// every pivot is positive.  limit_ns bounds every wait on an mbarrier.
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
  const float* Af = (const float*)(R + rg.Af);
  float* Lg = (float*)(R + rg.L);
  float* Linv_g = (float*)(R + rg.Linv);
  unsigned char* split_g = (unsigned char*)(R + rg.split);

  unsigned char* bufs = sm;
  float* LkT = (float*)(sm + 2 * kBufBytes);  // [panel][j * 32 + i] = L_kk(i, j)
  float* rdk = LkT + kMaxPanels * 1024;       // [panel][j] = 1 / L_kk(j, j)
  uint64_t* bars = (uint64_t*)(rdk + kMaxPanels * 32);  // [0] MMA done, [1], [2] bulk copies
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
  float shift = 0.0f;
  int attempt = 0;
  for (; attempt < 3 && result == 1; ++attempt) {
    shift = attempt == 0 ? 0.0f : (attempt == 1 ? 1e-5f : 1e-3f);
    if (tid == 0) sflag[1] = 0;
    __syncthreads();
    bool failed = false;
    for (int s = 0; s < S && !failed; ++s) {
      const int row = kSlab * s + tid;
      // this slab's rows of A~ (lower part, shifted diagonal) into tensor memory
      for (int c = 0; c < 4 * (s + 1); ++c) {
        float v[32];
        const float4* src = (const float4*)(Af + (((int64_t)s * P + c) * kSlab + tid) * kNb);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const float4 w = src[q];
          v[4 * q] = w.x;
          v[4 * q + 1] = w.y;
          v[4 * q + 2] = w.z;
          v[4 * q + 3] = w.w;
        }
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int col = kNb * c + j;
          v[j] = col < row ? v[j] : (col == row ? v[j] + shift : 0.0f);
        }
        tmem_st32(tlane + kNb * c, v);
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
        float* Lk = LkT + k * 1024;
        float* rk = rdk + k * 32;
        if (kd >= 0 && warp == kd) {
          // diagonal block: lane l holds row 32k + l; right-looking by columns with shuffles
          bool ok = true;
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const float ajj = __shfl_sync(0xffffffffu, a[j], j);
            ok = ok && ajj > 0.0f;
            const float rs = rsqrtf(ajj);
            const float lij = lane > j ? a[j] * rs : (lane == j ? ajj * rs : 0.0f);
            a[j] = lij;
            if (lane == j) rk[j] = rs;
#pragma unroll
            for (int m = j + 1; m < 32; ++m) a[m] = fmaf(-lij, __shfl_sync(0xffffffffu, lij, m), a[m]);
          }
#pragma unroll
          for (int m = 0; m < 32; ++m) Lk[m * 32 + lane] = a[m];
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
        // this row's entries of panel k: below the block, l L_kk^T = a by substitution
        if (row >= kNb * k + kNb) {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            a[j] *= rk[j];
            const float* col = Lk + j * 32;  // L_kk(m, j), m = 0..31
#pragma unroll
            for (int m4 = (j + 1) & ~3; m4 < 32; m4 += 4) {
              const float4 w = *(const float4*)(col + m4);
              if (m4 + 0 > j) a[m4 + 0] = fmaf(-a[j], w.x, a[m4 + 0]);
              if (m4 + 1 > j) a[m4 + 1] = fmaf(-a[j], w.y, a[m4 + 1]);
              if (m4 + 2 > j) a[m4 + 2] = fmaf(-a[j], w.z, a[m4 + 2]);
              if (m4 + 3 > j) a[m4 + 3] = fmaf(-a[j], w.w, a[m4 + 3]);
            }
          }
        } else if (row < kNb * k) {
#pragma unroll
          for (int m = 0; m < 32; ++m) a[m] = 0.0f;
        }
        if (row >= kNb * k) {
          float4* dst = (float4*)(Lg + (int64_t)row * np + kNb * k);
#pragma unroll
          for (int q = 0; q < 8; ++q) dst[q] = make_float4(a[4 * q], a[4 * q + 1], a[4 * q + 2], a[4 * q + 3]);
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
                const float x = a[8 * q + e + u];
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
        const int c0 = kNb * (k + 1), c1 = kSlab * (s + 1);
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
  if (result == 0) {
    // inverses of the diagonal blocks: lane j forms column j of L_kk^-1 by forward substitution
    for (int k = warp; k < P; k += kFactorThreads / 32) {
      const float* Lk = LkT + k * 1024;
      const float* rk = rdk + k * 32;
      float x[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        float acc = 0.0f;
#pragma unroll
        for (int m = 0; m < i; ++m) acc = fmaf(Lk[m * 32 + i], x[m], acc);
        x[i] = i < lane ? 0.0f : (i == lane ? rk[i] : -acc * rk[i]);
      }
#pragma unroll
      for (int i = 0; i < 32; ++i) Linv_g[(int64_t)k * 1024 + i * 32 + lane] = x[i];
    }
  }
  if (tid == 0) {
    hdr->fstat = result;
    hdr->attempts = attempt;
    hdr->shift = shift;
    const int64_t o = (int64_t)b * tb.stride;
    if (tb.ok) tb.ok[o] = result == 0 ? 1 : 0;
    if (tb.bad && result != 0) tb.bad[o] = 1;
  }
}

// X = L~^-1 by column panels, for the preconditioner's two products: CTA (j, b) forms the
// blocks of X(:, 32 j .. 32 j + 31) in turn,
//   X_jj = L_jj^-1,   X_kj = -L_kk^-1 sum_{m = j}^{k-1} L_km X_mj   (k > j),
// keeping them in shared memory, and writes each to X and, transposed, to XT (the blocks above
// the diagonal are never read).  For block k the row panel's blocks L_km, m = j .. k-1, are first
// copied to shared memory together (one memory latency per block); then the 256 threads form
// the sum as four groups (m = j + g, j + g + 4, ...) of 64 threads with a 4 x 4 tile each, the
// groups' tiles are added in group order, and the product with L_kk^-1 gives X_kj.
constexpr int kInvLd = 36;  // padded row stride of the shared 32 x 32 blocks
constexpr int kInverseSmem = (kMaxPanels * 1024 + (kMaxPanels - 1) * 32 * kInvLd + 5 * 32 * kInvLd) * 4;
__global__ void __launch_bounds__(256) k_tc_inverse(Batch tb) {
  extern __shared__ __align__(16) float ism[];
  float* Xs = ism;                              // [m][e * 32 + c]: X_mj
  float* Lb = Xs + kMaxPanels * 1024;           // [m - j][row * kInvLd + e]: L_km
  float* Tp = Lb + (kMaxPanels - 1) * 32 * kInvLd;  // [g][row * kInvLd + c]: group partials, then T
  const int j = blockIdx.x, b = blockIdx.y;
  if (b >= tb.B || !tb.on(b)) return;
  const int np = tb.np[b], P = np / kNb;
  if (j >= P) return;
  char* R = tb.base + tb.off[b];
  if (((const Hdr*)R)->fstat != 0) return;
  const Region rg = Region::of(np);
  const float* L = (const float*)(R + rg.L);
  const float* Linv = (const float*)(R + rg.Linv);
  float* X = (float*)(R + rg.X);
  float* XT = (float*)(R + rg.XT);
  const int t = threadIdx.x, g = t >> 6, tr = ((t & 63) >> 3) * 4, tc = (t & 7) * 4;
  for (int e = t; e < 1024; e += blockDim.x) {
    const float v = Linv[(int64_t)j * 1024 + e];
    const int ri = e / kNb, ci = e % kNb;
    Xs[j * 1024 + e] = v;
    X[(int64_t)(kNb * j + ri) * np + kNb * j + ci] = v;
    XT[(int64_t)(kNb * j + ci) * np + kNb * j + ri] = v;
  }
  for (int k = j + 1; k < P; ++k) {
    // L_km, m = j .. k-1 (rows 32k .. 32k + 31, columns 32 j .. 32 k - 1)
    const int nm = k - j;
    for (int e = t; e < nm * 32 * 8; e += blockDim.x) {
      const int mm = e / 256, ri = (e / 8) % 32, q = e % 8;
      const float4 v = *(const float4*)(L + (int64_t)(kNb * k + ri) * np + kNb * (j + mm) + 4 * q);
      *(float4*)(Lb + (mm * 32 + ri) * kInvLd + 4 * q) = v;
    }
    __syncthreads();
    float acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] = 0.0f;
    for (int mm = g; mm < nm; mm += 4) {
      const float* Lm = Lb + mm * 32 * kInvLd;
      const float* Xm = Xs + (j + mm) * 1024;
#pragma unroll 8
      for (int e = 0; e < 32; ++e) {
        const float4 x4 = *(const float4*)(Xm + e * 32 + tc);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float l = Lm[(tr + u) * kInvLd + e];
          acc[u][0] = fmaf(l, x4.x, acc[u][0]);
          acc[u][1] = fmaf(l, x4.y, acc[u][1]);
          acc[u][2] = fmaf(l, x4.z, acc[u][2]);
          acc[u][3] = fmaf(l, x4.w, acc[u][3]);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      *(float4*)(Tp + g * 32 * kInvLd + (tr + u) * kInvLd + tc) = make_float4(acc[u][0], acc[u][1], acc[u][2], acc[u][3]);
    __syncthreads();
    float* T = Tp + 4 * 32 * kInvLd;
    for (int e = t; e < 1024; e += blockDim.x) {
      const int ri = e / kNb, ci = e % kNb;
      float v = 0.0f;
#pragma unroll
      for (int gg = 0; gg < 4; ++gg) v += Tp[gg * 32 * kInvLd + ri * kInvLd + ci];
      T[ri * kInvLd + ci] = v;
    }
    __syncthreads();
    // X_kj = -L_kk^-1 T: thread t forms entries (t / 8, 4 (t % 8) .. + 3)
    {
      const int ri = t >> 3, c0 = (t & 7) * 4;
      const float* Li = Linv + (int64_t)k * 1024 + ri * 32;  // row ri of L_kk^-1
      float o[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll 8
      for (int e = 0; e <= ri; ++e) {
        const float le = Li[e];
        const float4 t4 = *(const float4*)(T + e * kInvLd + c0);
        o[0] = fmaf(le, t4.x, o[0]);
        o[1] = fmaf(le, t4.y, o[1]);
        o[2] = fmaf(le, t4.z, o[2]);
        o[3] = fmaf(le, t4.w, o[3]);
      }
      const float4 r4 = make_float4(-o[0], -o[1], -o[2], -o[3]);
      *(float4*)(Xs + k * 1024 + ri * 32 + c0) = r4;
      *(float4*)(X + (int64_t)(kNb * k + ri) * np + kNb * j + c0) = r4;
      XT[(int64_t)(kNb * j + c0 + 0) * np + kNb * k + ri] = r4.x;
      XT[(int64_t)(kNb * j + c0 + 1) * np + kNb * k + ri] = r4.y;
      XT[(int64_t)(kNb * j + c0 + 2) * np + kNb * k + ri] = r4.z;
      XT[(int64_t)(kNb * j + c0 + 3) * np + kNb * k + ri] = r4.w;
    }
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_factor(const Batch& tb, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(k_tc_factor, cudaFuncAttributeMaxDynamicSharedMemorySize, kFactorSmem);
  if (e != cudaSuccess) return e;
  k_tc_factor<<<tb.B, kFactorThreads, kFactorSmem, st>>>(tb, 1000000000ull);
  return cudaGetLastError();
}

cudaError_t launch_inverse(const Batch& tb, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(k_tc_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, kInverseSmem);
  if (e != cudaSuccess) return e;
  k_tc_inverse<<<dim3((unsigned)(tb.np_max / kNb), (unsigned)tb.B), 256, kInverseSmem, st>>>(tb);
  return cudaGetLastError();
}

}  // namespace tc
}  // namespace dnls
