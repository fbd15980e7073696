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
//            panel's diagonal block is factored in FP32 by one warp, the panel rows below it
//            solve L_ik L_kk^T = A_ik by substitution, and the trailing update A_ij -= L_ik L_jk^T is
//            issued as tcgen05.mma (kind::f16, BF16 operands, FP32 accumulation) on the 3-term
//            BF16 split x = x0 + x1 + x2 of the FP32 panel (products x0y0 + x0y1 + x1y0 + x0y2 +
//            x1y1 + x2y0, which keeps FP32-level accuracy: Henry, Tang & Heinecke, "Leveraging
//            the bfloat16 artificial intelligence datatype for higher-precision computations",
//            ARITH 2019).  Slabs are taken in turn (left-looking over slabs, right-looking inside
//            one): the rows of earlier slabs enter a later slab's updates as MMA B operands,
//            copied from a global staging area into shared memory with cp.async.bulk.
//   inverse  X = L~^-1 in FP32 by 32-column panels (one CTA per problem and panel), stored with
//            its transpose, so that applying M^-1 = X^T X is two dense products
//   solve    preconditioned conjugate gradients in FP64 on A~ x~ = D b with M = L~ L~^T, then
//            x = D x~.  A thread-block cluster per problem: each CTA owns a block of rows and
//            forms their part of the FP64 product with A~ and of the two FP32 products with X.
//            With max_steps = 0 the call applies M^-1 once (a preconditioner).
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
constexpr int kPcgThreads = 384;  // = kMaxN: one thread per (row, K-split) of a CTA's rows
constexpr int kMaxCluster = 8;
// shared memory of the factor kernel: two panel buffers, the diagonal blocks L_kk (transposed)
// and their reciprocal pivots, three mbarriers, the tensor-memory address slot and two flags
constexpr int kFactorSmem = 2 * kBufBytes + kMaxPanels * 1024 * 4 + kMaxPanels * 32 * 4 + 64;

// Per-problem header at the start of its region.
constexpr int kHdrBytes = 512;
enum { kPartB = 0, kPartPQ, kPartRR, kPartRZ, kParts };
struct Hdr {
  int32_t fstat;      // factor: 0 ok, 1 not positive definite after every shift, 2 timeout
  int32_t steps;      // PCG steps of the last solve
  int32_t attempts;   // factor: shifts tried
  int32_t pad;
  double resid;       // PCG: final ||b~ - A~ x~|| / ||b~|| (recurrence residual)
  double shift;       // factor: the diagonal shift that succeeded
  // per-CTA partials of the cluster's reductions, one slot array per quantity (a slot is
  // rewritten only two cluster barriers after it was read)
  double part[kParts][kMaxCluster];
};
static_assert(sizeof(Hdr) <= kHdrBytes, "header");

__host__ __device__ inline int64_t a256(int64_t x) { return (x + 255) & ~(int64_t)255; }

// Byte offsets of a problem's arrays inside its region, for padded order np.
//   A    FP64 scaled matrix, row-major (the CG products)
//   Af   the same in FP32, chunk-major: chunk (s, c) = rows 128 s .. 128 s + 127, columns
//        32 c .. 32 c + 31, each row's 32 values contiguous (coalesced slab loads of the factor)
//   L    FP32 factor, row-major (lower triangle)       Linv  FP32 inverted diagonal blocks
//   X    FP32 L~^-1, row-major (lower triangle), and XT its transpose, row-major: the
//        preconditioner's two products read them with consecutive threads on consecutive rows
//   split  BF16 split panels (MMA B operands of later slabs)    vec  CG vectors
struct Region {
  int64_t d, A, Af, L, Linv, X, XT, split, vec, bytes;
  __host__ __device__ static Region of(int np) {
    Region r;
    int64_t o = kHdrBytes;
    r.d = o;
    o = a256(o + (int64_t)np * 8);
    r.A = o;
    o = a256(o + (int64_t)np * np * 8);
    r.Af = o;
    o = a256(o + (int64_t)np * np * 4);
    r.L = o;
    o = a256(o + (int64_t)np * np * 4);
    r.Linv = o;
    o = a256(o + (int64_t)(np / kNb) * 1024 * 4);
    r.X = o;
    o = a256(o + (int64_t)np * np * 4);
    r.XT = o;
    o = a256(o + (int64_t)np * np * 4);
    r.split = o;
    o = a256(o + (int64_t)(np / kNb) * 3 * np * 64);
    r.vec = o;  // p (FP64), r (FP32, scaled), y (FP32)
    o = a256(o + (int64_t)np * 16);
    r.bytes = o;
    return r;
  }
};

// The problems of one call: region b starts at base + off[b]; np[b] = 0 skips a problem, as does
// active[b * stride] == 0 when `active` is set.  On a failed factorization ok[b * stride] = 0 and
// bad[b * stride] = 1 are written where those pointers are set (ok = 1 on success).
struct Batch {
  int B;
  int np_max;  // largest np (host side: grid sizes)
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
  float* Af = (float*)(R + rg.Af);
  const int s = r0 / kSlab, P = np / kNb;
  for (int e = threadIdx.x; e < kNb * np; e += blockDim.x) {
    const int i = r0 + e / np, j = e % np;
    double v;
    if (i < n && j < n) v = (j <= i ? src.val(b, i, j) : src.val(b, j, i)) * ds[i] * ds[j];
    else v = i == j ? 1.0 : 0.0;
    A[(int64_t)i * np + j] = v;
    Af[(((int64_t)s * P + j / kNb) * kSlab + (i % kSlab)) * kNb + j % kNb] = (float)v;
  }
  if (blockIdx.x == 0) {
    double* d = (double*)(R + rg.d);
    for (int i = threadIdx.x; i < np; i += blockDim.x) d[i] = ds[i];
  }
}

// ----------------------------------------------------------------------------- factor
// One CTA of kFactorThreads per active problem (dnls_tc.cu): L~ into the region's L / Linv;
// launch_inverse then forms X = L~^-1 and X^T (one CTA per problem and 32-column panel).
// Errors surface through the returned launch status.
cudaError_t launch_factor(const Batch& tb, cudaStream_t st);
cudaError_t launch_inverse(const Batch& tb, cudaStream_t st);

// ----------------------------------------------------------------------------- solve
// Sum (or max) over the CTA in a fixed order: warp shuffles, then every thread adds the warps'
// partials from shared memory `red` (>= 32 doubles).  Two barriers.
__device__ __forceinline__ double cta_reduce(double v, double* red, bool is_max) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double w = __shfl_xor_sync(0xffffffffu, v, o);
    v = is_max ? fmax(v, w) : v + w;
  }
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = red[0];
  for (int i = 1; i < nw; ++i) t = is_max ? fmax(t, red[i]) : t + red[i];
  __syncthreads();
  return t;
}

// Barrier over the problem's kc CTAs (a thread-block cluster), with release / acquire at
// cluster scope so that every global write before it is visible after it.
__device__ __forceinline__ void pcg_sync(int kc) {
  if (kc > 1) cluster_sync_all();
  else __syncthreads();
}

// Cluster-wide reduction: each CTA publishes its partial in slot `kind`, and after the barrier
// (whose acquire makes the other CTAs' writes visible) every CTA adds the kc partials in rank
// order, the same value in every CTA.
__device__ __forceinline__ double cluster_total(Hdr* hdr, int kind, int rank, int kc, double part, bool is_max) {
  if (threadIdx.x == 0) hdr->part[kind][rank] = part;
  pcg_sync(kc);
  double v[kMaxCluster];
#pragma unroll
  for (int c = 0; c < kMaxCluster; ++c) v[c] = c < kc ? __ldcg(&hdr->part[kind][c]) : 0.0;
  double t = v[0];
  for (int c = 1; c < kc; ++c) t = is_max ? fmax(t, v[c]) : t + v[c];
  return t;
}

// Two sums over the CTA at once (fixed order, as cta_reduce).
__device__ __forceinline__ void cta_reduce2(double& a, double& c, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
  }
  if (lane == 0) {
    red[warp] = a;
    red[32 + warp] = c;
  }
  __syncthreads();
  double ta = red[0], tc = red[32];
  for (int i = 1; i < nw; ++i) {
    ta += red[i];
    tc += red[32 + i];
  }
  __syncthreads();
  a = ta;
  c = tc;
}

// Preconditioned conjugate gradients on A~ x~ = b~ (b~ = D b) with M^-1 = X^T X, X = L~^-1;
// kc CTAs per problem in one thread-block cluster (kc divides np / 32), CTA c owning rows
// [c np / kc, (c + 1) np / kc).  Thread t < rows keeps x, r, p, z of row row0 + t in registers;
// for the products thread t works on row row0 + t % rows over the column split t / rows
// (nsplit = 384 / rows splits), and the split partials are added by the row's thread in split
// order.  Per step: q = A~ p on own rows (FP64; A~ is symmetric, so row i is read as column i,
// consecutive threads on consecutive addresses), alpha, x, r; y = X r on own rows (reading X^T)
// and z = X^T y on own entries (reading X), FP32 with r scaled by the last ||r||; r.r and r.z in
// one reduction; beta, p.  The cluster exchanges p, r and y through the region and its scalars
// through the header's partial slots, five cluster barriers per step; every CTA takes the same
// stop decision.
//   IO::rhs_of(b, i)         b_i of the original system (i < n)
//   IO::n(b)                 the order
//   IO::out(b, i, x_i)       the solution (i < n), written once converged or stopped
//   IO::report(b, steps, resid, ok)   per-problem outcome (ok false: a breakdown, p'Ap <= 0)
//   IO::factor_failed(b, fstat)       the factor failed (1) or timed out (2): nothing solved
// max_steps = 0 applies M^-1 once (x = D X^T X D b).
template <class IO>
__global__ void __launch_bounds__(kPcgThreads, 1) k_tc_pcg(Batch tb, IO io, int max_steps, double tol, int kc) {
  __shared__ double ps[kMaxN];                 // p, staged for the product
  __shared__ float vs[kMaxN];                  // scaled r, then y, staged for the preconditioner
  __shared__ double qpart[kPcgThreads];        // split partials of the row products
  __shared__ float fpart[kPcgThreads];
  __shared__ double red[64];
  const int b = blockIdx.x / kc, rank = blockIdx.x % kc;
  if (b >= tb.B || !tb.on(b)) return;  // the same for every CTA of the cluster
  const int np = tb.np[b];
  char* R = tb.base + tb.off[b];
  Hdr* hdr = (Hdr*)R;
  if (hdr->fstat != 0) {  // written by the factor launch; the same for the whole cluster
    if (rank == 0 && threadIdx.x == 0) io.factor_failed(b, hdr->fstat);
    return;
  }
  const Region rg = Region::of(np);
  const double* A = (const double*)(R + rg.A);
  const double* d = (const double*)(R + rg.d);
  const float* X = (const float*)(R + rg.X);
  const float* XT = (const float*)(R + rg.XT);
  double* vp = (double*)(R + rg.vec);
  float* vr = (float*)(vp + np);
  float* vy = vr + np;
  const int tid = threadIdx.x;
  const int n = io.n(b);
  const int rows = np / kc, row0 = rank * rows;
  const int nsplit = kPcgThreads / rows < 1 ? 1 : kPcgThreads / rows;
  const int width = (np + nsplit - 1) / nsplit;
  const int pr = row0 + tid % rows, sp = tid / rows;          // product row and split
  const bool pact = sp < nsplit;
  const int j0 = sp * width, j1 = j0 + width < np ? j0 + width : np;
  const bool own = tid < rows;
  const int ir = row0 + tid;                                    // own row
  // q_pr = sum_j A~(j, pr) p_j over this thread's split, then summed per own row
  auto rows_fp64 = [&]() -> double {
    double a4[4] = {0.0, 0.0, 0.0, 0.0};
    if (pact) {
      const double* Ac = A + pr;
      int j = j0;
      for (; j + 8 <= j1; j += 8) {
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = __ldg(Ac + (int64_t)(j + u) * np);
#pragma unroll
        for (int u = 0; u < 8; ++u) a4[u & 3] = fma(v[u], ps[j + u], a4[u & 3]);
      }
      for (; j < j1; ++j) a4[0] = fma(__ldg(Ac + (int64_t)j * np), ps[j], a4[0]);
    }
    const double acc = (a4[0] + a4[1]) + (a4[2] + a4[3]);
    qpart[tid] = acc;
    __syncthreads();
    double q = 0.0;
    if (own)
      for (int s = 0; s < nsplit; ++s) q += qpart[s * rows + tid];
    __syncthreads();
    return q;
  };
  // z = X^T X r for the own row, r given scaled by 1 / sc
  auto precond = [&](double rv, double sc) -> double {
    if (own) vr[ir] = (float)(rv / sc);
    pcg_sync(kc);
    for (int i = tid; i < np; i += kPcgThreads) vs[i] = vr[i];
    __syncthreads();
    // y_pr = sum_{j <= pr} X(pr, j) r_j, and below z_pr = sum_{i >= pr} X(i, pr) y_i: column
    // sums over [lo, hi) of a row-major matrix M, 16 loads in flight per thread
    auto colsum = [&](const float* M, int lo, int hi) -> float {
      float f4[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      const float* Mc = M + pr;
      int j = lo;
      for (; j + 16 <= hi; j += 16) {
        float v[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) v[u] = __ldg(Mc + (int64_t)(j + u) * np);
#pragma unroll
        for (int u = 0; u < 16; ++u) f4[u & 3] = fmaf(v[u], vs[j + u], f4[u & 3]);
      }
      for (; j < hi; ++j) f4[0] = fmaf(__ldg(Mc + (int64_t)j * np), vs[j], f4[0]);
      return (f4[0] + f4[1]) + (f4[2] + f4[3]);
    };
    float acc = 0.0f;
    if (pact) acc = colsum(XT, j0, j1 < pr + 1 ? j1 : pr + 1);
    fpart[tid] = acc;
    __syncthreads();
    if (own) {
      float y = 0.0f;
      for (int s = 0; s < nsplit; ++s) y += fpart[s * rows + tid];
      vy[ir] = y;
    }
    pcg_sync(kc);
    for (int i = tid; i < np; i += kPcgThreads) vs[i] = vy[i];
    __syncthreads();
    acc = 0.0f;
    if (pact) acc = colsum(X, j0 > pr ? j0 : pr, j1);
    fpart[tid] = acc;
    __syncthreads();
    float z = 0.0f;
    if (own)
      for (int s = 0; s < nsplit; ++s) z += fpart[s * rows + tid];
    __syncthreads();
    return own ? (double)z * sc : 0.0;
  };
  double x = 0.0, r = own && ir < n ? io.rhs_of(b, ir) * d[ir] : 0.0, p = 0.0, z = 0.0;
  const double bn = sqrt(cluster_total(hdr, kPartB, rank, kc, cta_reduce(r * r, red, false), false));
  int steps = 0;
  double rn = bn;
  bool ok = true;
  if (bn > 0.0) {
    z = precond(r, bn);
    double rz = cluster_total(hdr, kPartRZ, rank, kc, cta_reduce(r * z, red, false), false);
    if (max_steps <= 0) x = z;
    p = z;
    while (steps < max_steps) {
      if (own) vp[ir] = p;
      pcg_sync(kc);
      for (int i = tid; i < np; i += kPcgThreads) ps[i] = vp[i];
      __syncthreads();
      const double q = rows_fp64();
      const double pq = cluster_total(hdr, kPartPQ, rank, kc, cta_reduce(p * q, red, false), false);
      const double alpha = rz / pq;
      ++steps;
      if (!(pq > 0.0) || !isfinite(alpha)) {
        ok = false;
        break;
      }
      x += alpha * p;
      r -= alpha * q;
      z = precond(r, rn);
      double rr = r * r, rz2 = r * z;
      cta_reduce2(rr, rz2, red);
      if (threadIdx.x == 0) {
        hdr->part[kPartRR][rank] = rr;
        hdr->part[kPartRZ][rank] = rz2;
      }
      pcg_sync(kc);
      {
        double v1[kMaxCluster], v2[kMaxCluster];
#pragma unroll
        for (int c = 0; c < kMaxCluster; ++c) {
          v1[c] = c < kc ? __ldcg(&hdr->part[kPartRR][c]) : 0.0;
          v2[c] = c < kc ? __ldcg(&hdr->part[kPartRZ][c]) : 0.0;
        }
        rr = v1[0];
        rz2 = v2[0];
        for (int c = 1; c < kc; ++c) {
          rr += v1[c];
          rz2 += v2[c];
        }
      }
      rn = sqrt(rr);
      if (!(rn > tol * bn) || steps >= max_steps) break;
      const double beta = rz2 / rz;
      rz = rz2;
      p = z + beta * p;
    }
  }
  if (own && ir < n) io.out(b, ir, x * d[ir]);
  if (rank == 0 && tid == 0) {
    const double res = bn > 0.0 ? rn / bn : 0.0;
    hdr->steps = steps;
    hdr->resid = res;
    io.report(b, steps, res, ok);
  }
}

// Launch of the solve, shared with the bundle-adjustment path.
template <class IO>
inline cudaError_t launch_pcg(const Batch& tb, const IO& io, int steps, double tol, int kc, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(tb.B * kc));
  cfg.blockDim = dim3(kPcgThreads);
  cfg.dynamicSmemBytes = 0;
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
