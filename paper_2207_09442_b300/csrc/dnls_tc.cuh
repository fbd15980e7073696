// Dense batched SPD solves with a tensor-core Cholesky factor and FP64 refinement, for the dense
// reduced camera systems of bundle adjustment (Sec. 4.2: the point blocks are eliminated by the
// Schur complement and the reduced problem goes to a Cholesky solver) and for plain batches of
// dense SPD matrices.
//
// Per problem (order n, padded to np = 128 * S, S <= 3):
//   densify  A~ = D A D with D = diag(2^-floor(log2(A_ii)/2)) (exact power-of-two scaling, so the
//            FP64 scaled system is the original one; diagonal in [1, 4)), FP64 row-major np x np
//   factor   L~ L~^T = A~ (+ sigma I on retry) in FP32: right-looking by 32-wide panels; the
//            128-row slab being factored lives in tensor memory as an FP32 accumulator, each
//            panel's diagonal block is factored and inverted in FP32 by one warp, the panel rows
//            below it are L_ik = A_ik L_kk^-T, and the trailing update A_ij -= L_ik L_jk^T is
//            issued as tcgen05.mma (kind::f16, BF16 operands, FP32 accumulation) on the 3-term
//            BF16 split x = x0 + x1 + x2 of the FP32 panel (products x0y0 + x0y1 + x1y0 + x0y2 +
//            x1y1 + x2y0, which keeps FP32-level accuracy: Henry, Tang & Heinecke, "Leveraging
//            the bfloat16 artificial intelligence datatype for higher-precision computations",
//            ARITH 2019).  Slabs are taken in turn (left-looking over slabs, right-looking inside
//            one): the rows of earlier slabs enter a later slab's updates as MMA B operands,
//            copied from a global staging area into shared memory with cp.async.bulk.
//   solve    preconditioned conjugate gradients in FP64 on A~ x~ = D b with M = L~ L~^T
//            (FP32 triangular solves), then x = D x~.  A thread-block cluster per problem: every
//            CTA multiplies its rows of A~ (FP64), CTA 0 runs the updates and the triangular
//            solves.  With max_steps = 0 the call applies M^-1 once (a preconditioner).
//
// Operand layout for tcgen05.mma (K-major, no swizzle): a 32-column BF16 panel of R rows is
// stored as core matrices of 8 rows x 16 bytes; the core matrix of row group g and K chunk q
// (8 columns) sits at g * 512 + q * 128 bytes, so LBO (K direction) = 128 B and SBO (8-row
// groups) = 512 B; K step kk of an MMA (16 columns) starts kk * 256 bytes further.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "dnls_blockchol.cuh"  // block_sum, cluster_sync_all

namespace dnls {
namespace tc {

constexpr int kNb = 32;                         // panel width
constexpr int kSlab = 128;                      // rows of one tensor-memory accumulator (MMA M)
constexpr int kMaxN = 384;                      // largest padded order (shared-memory budget)
constexpr int kMaxPanels = kMaxN / kNb;
constexpr int kTermBytes = kMaxN / 8 * 512;     // one BF16 split term of a panel, all rows
constexpr int kBufBytes = 3 * kTermBytes;       // the three split terms
constexpr int kFactorThreads = 128;             // warp w owns tensor-memory lanes 32w..32w+31
constexpr int kPcgThreads = 256;
constexpr int kMaxCluster = 8;
// shared memory of the factor kernel: two panel buffers, the inverted diagonal blocks, the
// diagonal-block scratch (32 x 33) and its reciprocal pivots, three mbarriers, the tensor-memory
// address slot and two flags
constexpr int kFactorSmem = 2 * kBufBytes + kMaxPanels * 1024 * 4 + 32 * 33 * 4 + 32 * 4 + 64;

// Per-problem header at the start of its region.
struct Hdr {
  int32_t fstat;      // factor: 0 ok, 1 not positive definite after every shift, 2 timeout
  int32_t steps;      // PCG steps of the last solve (-1: not run)
  int32_t done;       // PCG: converged or stopped (shared by the cluster)
  int32_t attempts;   // factor: shifts tried
  double resid;       // PCG: final ||b~ - A~ x~|| / ||b~||
  double bnorm, rz, shift, alpha;
  double part[kMaxCluster];  // per-CTA partial dot products
};
static_assert(sizeof(Hdr) <= 256, "header");

__host__ __device__ inline int64_t a256(int64_t x) { return (x + 255) & ~(int64_t)255; }

// Byte offsets of a problem's arrays inside its region, for padded order np.
struct Region {
  int64_t d, A, L, Linv, split, vec, bytes;
  __host__ __device__ static Region of(int np) {
    Region r;
    int64_t o = 256;
    r.d = o;
    o = a256(o + (int64_t)np * 8);
    r.A = o;
    o = a256(o + (int64_t)np * np * 8);
    r.L = o;
    o = a256(o + (int64_t)np * np * 4);
    r.Linv = o;
    o = a256(o + (int64_t)(np / kNb) * 1024 * 4);
    r.split = o;
    o = a256(o + (int64_t)(np / kNb) * 3 * np * 64);
    r.vec = o;  // b, x, r, z, p, q
    o = a256(o + (int64_t)6 * np * 8);
    r.bytes = o;
    return r;
  }
};

// The problems of one call: region b starts at base + off[b]; np[b] = 0 skips a problem, as does
// active[b * stride] == 0 when `active` is set.  On a failed factorization ok[b * stride] = 0 and
// bad[b * stride] = 1 are written where those pointers are set (ok = 1 on success).
struct Batch {
  int B;
  char* base;
  const int64_t* off;
  const int32_t* np;
  const int32_t* active;
  int32_t* ok;
  int32_t* bad;
  int stride;
  __device__ bool on(int b) const {
    return np[b] > 0 && (active == nullptr || active[(int64_t)b * stride] != 0);
  }
};

// ----------------------------------------------------------------------------- PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for the phase of the given parity to complete, for at most limit_ns nanoseconds.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait(bar, parity))
    if (global_ns() - t0 > limit_ns) return false;
  return true;
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// 1-D bulk copy global -> shared (this CTA), completing `bytes` on the mbarrier
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// whole warp
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
// 32 consecutive FP32 columns of this thread's tensor-memory lane (warp-wide), waited for
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
      "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "
      "[%32];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const float* v) {
  uint32_t r[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) r[i] = __float_as_uint(v[i]);
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
      "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, "
      "%32};\n"
      "tcgen05.wait::st.sync.aligned;\n" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
      "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]),
      "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]),
      "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
      : "memory");
}
// shared-memory matrix descriptor: K-major, no swizzle, LBO / SBO in bytes, version 1
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         (1ull << 46);
}
// instruction descriptor, kind::f16: D FP32, A and B BF16, both K-major, A negated, M = 128
__host__ __device__ constexpr uint32_t idesc_bf16_negA(int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (1u << 13) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
// D[tmem] = -A B^T + D (accumulate) on this CTA's tensor core
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(1u)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// ----------------------------------------------------------------------------- densify
// A~ = D A D (FP64, np x np, identity on the padding) and D for every active problem.
// Src::n(b) is the order, Src::val(b, i, j) the FP64 entry A_ij (i, j < n; only i >= j is asked
// for: the kernel mirrors it).  grid (np_max / 32, B): CTA (strip, b) writes rows 32 strip ...
template <class Src>
__global__ void __launch_bounds__(256) k_tc_densify(Batch tb, Src src) {
  __shared__ double ds[kMaxN];
  const int b = blockIdx.y;
  if (b >= tb.B || !tb.on(b)) return;
  const int np = tb.np[b], n = src.n(b);
  const int r0 = blockIdx.x * kNb;
  if (r0 >= np) return;
  char* R = tb.base + tb.off[b];
  const Region rg = Region::of(np);
  for (int i = threadIdx.x; i < np; i += blockDim.x) {
    double s = 1.0;
    if (i < n) {
      const double a = src.val(b, i, i);
      // 2^-floor(e/2) with a in [2^e, 2^(e+1)): exact, a s^2 in [1, 4)
      if (a > 0.0 && isfinite(a)) s = ldexp(1.0, -(ilogb(a) >> 1));
    }
    ds[i] = s;
  }
  __syncthreads();
  double* A = (double*)(R + rg.A);
  for (int e = threadIdx.x; e < kNb * np; e += blockDim.x) {
    const int i = r0 + e / np, j = e % np;
    double v;
    if (i < n && j < n) v = (j <= i ? src.val(b, i, j) : src.val(b, j, i)) * ds[i] * ds[j];
    else v = i == j ? 1.0 : 0.0;
    A[(int64_t)i * np + j] = v;
  }
  if (blockIdx.x == 0) {
    double* d = (double*)(R + rg.d);
    for (int i = threadIdx.x; i < np; i += blockDim.x) d[i] = ds[i];
  }
}

// ----------------------------------------------------------------------------- factor
// One CTA of kFactorThreads per active problem (dnls_tc.cu): L~ into the region's L / Linv.
// Errors surface through the returned launch status.
cudaError_t launch_factor(const Batch& tb, cudaStream_t st);

// ----------------------------------------------------------------------------- solve
// z = M^-1 r in FP32 (y = L~^-1 r, z = L~^-T y), one CTA: ys (shared, np floats) holds r on entry
// and z on exit; Linv_s the staged inverted diagonal blocks; L row-major FP32.
__device__ inline void tc_precond(float* ys, const float* Linv_s, const float* L, int np, float* tmp) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int P = np / kNb;
  for (int k = 0; k < P; ++k) {
    const int base = k * kNb;
    if (tid < 32) {
      const float* Li = Linv_s + k * 1024 + tid * 32;
      float acc = 0.0f;
#pragma unroll
      for (int m = 0; m < 32; ++m) acc = fmaf(m <= tid ? Li[m] : 0.0f, ys[base + m], acc);
      tmp[tid] = acc;
    }
    __syncthreads();
    if (tid < 32) ys[base + tid] = tmp[tid];
    for (int i = base + kNb + tid; i < np; i += nt) {
      const float4* Lr = (const float4*)(L + (int64_t)i * np + base);
      float acc = 0.0f;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float4 w = Lr[q];
        acc = fmaf(w.x, tmp[4 * q], fmaf(w.y, tmp[4 * q + 1], fmaf(w.z, tmp[4 * q + 2], fmaf(w.w, tmp[4 * q + 3], acc))));
      }
      ys[i] -= acc;
    }
    __syncthreads();
  }
  for (int k = P - 1; k >= 0; --k) {
    const int base = k * kNb;
    if (tid < 32) {
      float acc = 0.0f;
#pragma unroll
      for (int m = 0; m < 32; ++m) acc = fmaf(m >= tid ? Linv_s[k * 1024 + m * 32 + tid] : 0.0f, ys[base + m], acc);
      tmp[tid] = acc;
    }
    __syncthreads();
    if (tid < 32) ys[base + tid] = tmp[tid];
    for (int j = tid; j < base; j += nt) {
      float acc = 0.0f;
#pragma unroll 8
      for (int m = 0; m < 32; ++m) acc = fmaf(L[(int64_t)(base + m) * np + j], tmp[m], acc);
      ys[j] -= acc;
    }
    __syncthreads();
  }
}

// Preconditioned conjugate gradients on A~ x~ = b~ (b~ = D b), M = L~ L~^T; kc CTAs per problem
// in one thread-block cluster (kc in 1, 2, 4, 8; np / kc rows of the product each).
//   IO::rhs_of(b, i)         b_i of the original system (i < n)
//   IO::n(b)                 the order
//   IO::out(b, i, x_i)       the solution (i < n), written once converged or stopped
//   IO::report(b, steps, resid, ok)   per-problem outcome (ok false: a breakdown, p'Ap <= 0)
// max_steps = 0 applies M^-1 once (x = D M^-1 D b).
// Dynamic shared memory: kPcgSmem (the staged inverted diagonal blocks).
constexpr int kPcgSmem = kMaxPanels * 1024 * 4;
template <class IO>
__global__ void __launch_bounds__(kPcgThreads) k_tc_pcg(Batch tb, IO io, int max_steps, double tol, int kc) {
  __shared__ double ps[kMaxN];
  __shared__ float ys[kMaxN];
  __shared__ float tmp[32];
  __shared__ double red[kPcgThreads];
  extern __shared__ __align__(16) float Linv_s[];
  const int b = blockIdx.x / kc, rank = blockIdx.x % kc;
  if (b >= tb.B || !tb.on(b)) return;  // the same for every CTA of the cluster
  const int np = tb.np[b];
  char* R = tb.base + tb.off[b];
  Hdr* hdr = (Hdr*)R;
  if (hdr->fstat != 0) return;  // written by the factor launch; the same for the whole cluster
  const Region rg = Region::of(np);
  const double* A = (const double*)(R + rg.A);
  const double* d = (const double*)(R + rg.d);
  const float* L = (const float*)(R + rg.L);
  double* vb = (double*)(R + rg.vec);
  double *vx = vb + np, *vr = vb + 2 * np, *vz = vb + 3 * np, *vp = vb + 4 * np, *vq = vb + 5 * np;
  const int tid = threadIdx.x;
  const int n = io.n(b);
  // M^-1 applied to vr into vz (rank 0), r scaled by its largest entry for the FP32 sweeps
  auto precond = [&]() {
    double mx = 0.0;
    for (int i = tid; i < np; i += blockDim.x) mx = fmax(mx, fabs(vr[i]));
    // block max through the sum buffer
    red[tid] = mx;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if (tid < w) red[tid] = fmax(red[tid], red[tid + w]);
      __syncthreads();
    }
    const double sc = red[0] > 0.0 ? red[0] : 1.0;
    __syncthreads();
    for (int i = tid; i < np; i += blockDim.x) ys[i] = (float)(vr[i] / sc);
    __syncthreads();
    tc_precond(ys, Linv_s, L, np, tmp);
    for (int i = tid; i < np; i += blockDim.x) vz[i] = (double)ys[i] * sc;
    __syncthreads();
  };
  if (rank == 0) {
    const float* Lig = (const float*)(R + rg.Linv);
    for (int i = tid; i < (np / kNb) * 1024; i += blockDim.x) Linv_s[i] = Lig[i];
    double acc = 0.0;
    for (int i = tid; i < np; i += blockDim.x) {
      const double v = i < n ? io.rhs_of(b, i) * d[i] : 0.0;
      vb[i] = v;
      vr[i] = v;
      vx[i] = 0.0;
      acc += v * v;
    }
    const double bn = sqrt(block_sum(acc, red));
    precond();
    double rz = 0.0;
    for (int i = tid; i < np; i += blockDim.x) {
      vp[i] = vz[i];
      rz += vr[i] * vz[i];
    }
    rz = block_sum(rz, red);
    if (tid == 0) {
      hdr->bnorm = bn;
      hdr->rz = rz;
      hdr->steps = 0;
      hdr->resid = bn > 0.0 ? 1.0 : 0.0;
      hdr->done = (max_steps <= 0 || !(bn > 0.0)) ? 1 : 0;
    }
    if (max_steps <= 0)
      for (int i = tid; i < np; i += blockDim.x) vx[i] = vz[i];
  }
  if (kc > 1) cluster_sync_all();
  else __syncthreads();
  bool ok = true;
  const int rows = np / kc, row0 = rank * rows;
  const int warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
  for (int it = 0;; ++it) {
    if (*(volatile int32_t*)&hdr->done) break;
    for (int i = tid; i < np; i += blockDim.x) ps[i] = vp[i];
    __syncthreads();
    double part = 0.0;
    for (int i = row0 + warp; i < row0 + rows; i += nw) {
      const double* Ai = A + (int64_t)i * np;
      double acc = 0.0;
      for (int j = lane; j < np; j += 32) acc = fma(Ai[j], ps[j], acc);
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
      if (lane == 0) {
        vq[i] = acc;
        part += acc * ps[i];
      }
    }
    part = block_sum(part, red);
    if (tid == 0) hdr->part[rank] = part;
    if (kc > 1) cluster_sync_all();
    else __syncthreads();
    if (rank == 0) {
      double pq = 0.0;
      for (int c = 0; c < kc; ++c) pq += *(volatile double*)&hdr->part[c];
      const double rz = hdr->rz;
      const double alpha = rz / pq;
      const bool good = pq > 0.0 && isfinite(alpha);
      double r2 = 0.0;
      if (good)
        for (int i = tid; i < np; i += blockDim.x) {
          vx[i] += alpha * vp[i];
          vr[i] -= alpha * vq[i];
          r2 += vr[i] * vr[i];
        }
      const double rn = sqrt(block_sum(r2, red));
      const double bn = hdr->bnorm;
      const bool stop = !good || !(rn > tol * bn) || it + 1 >= max_steps;
      if (!stop) {
        precond();
        double rz2 = 0.0;
        for (int i = tid; i < np; i += blockDim.x) rz2 += vr[i] * vz[i];
        rz2 = block_sum(rz2, red);
        const double beta = rz2 / rz;
        for (int i = tid; i < np; i += blockDim.x) vp[i] = vz[i] + beta * vp[i];
        if (tid == 0) hdr->rz = rz2;
      }
      if (tid == 0) {
        hdr->steps = it + 1;
        if (good) hdr->resid = rn / bn;
        hdr->done = stop ? 1 : 0;
      }
      if (!good) ok = false;
    }
    if (kc > 1) cluster_sync_all();
    else __syncthreads();
  }
  if (rank == 0) {
    for (int i = tid; i < n; i += blockDim.x) io.out(b, i, vx[i] * d[i]);
    if (tid == 0) io.report(b, hdr->steps, hdr->resid, ok);
  }
}

// Launch of the solve, shared with the bundle-adjustment path.
template <class IO>
inline cudaError_t launch_pcg(const Batch& tb, const IO& io, int steps, double tol, int kc, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(k_tc_pcg<IO>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPcgSmem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(tb.B * kc));
  cfg.blockDim = dim3(kPcgThreads);
  cfg.dynamicSmemBytes = kPcgSmem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)kc;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = kc > 1 ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k_tc_pcg<IO>, tb, io, steps, tol, kc);
}


}  // namespace tc
}  // namespace dnls
