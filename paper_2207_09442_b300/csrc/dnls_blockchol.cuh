// Level-scheduled, left-looking block Cholesky of a block-sparse SPD matrix and the matching
// triangular solves, run by one CTA or by the CTAs of a thread-block cluster (Sec. 4.2's sparse
// Cholesky with a symbolic factorization computed once per structure).  The view type F supplies
// the symbolic structure and buffers (fields N, nnzL, nlev, chain_lev, dense_lev, H, L, Linv,
// tmp, lsrc, tgtptr, tgt, gptr, gsrc, gsplit, lvlptr, lvlcols, panptr, pan, rowptr, rowent,
// rsplit, colptr, rows, glanes, slanes; see ProbMeta in dnls_graph.h for their meaning).
// Every output element is produced by one thread in a fixed order: no atomics, bitwise
// reproducible results.
#pragma once

#include <cuda_runtime.h>

namespace dnls {

constexpr double kDiagFloor = 1e-9;
// sum over each group of `lanes` adjacent lanes (a power of two <= 8), same fixed order in
// every lane; `lanes` must be the same for the whole warp, and all its lanes must call this
__device__ __forceinline__ double lane_sum(double v, int lanes) {
  for (int o = 1; o < lanes; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float lane_sum(float v, int lanes) {
  for (int o = 1; o < lanes; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }

// ----------------------------------------------------------------------------- helpers
// Thread-block cluster barrier with release / acquire semantics at cluster scope: every write
// (shared or global) of every thread of the cluster before it is visible to every thread after it.
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

// One value of CTA `rank`'s shared memory at the offset of `local` (distributed shared memory of
// the thread-block cluster).
__device__ __forceinline__ int ld_cluster_shared(const int* local, int rank) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(local);
  uint32_t ra;
  int v;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
  asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(ra) : "memory");
  return v;
}
__device__ __forceinline__ double ld_cluster_shared(const double* local, int rank) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(local);
  uint32_t ra;
  double v;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(ra) : "memory");
  return v;
}

__device__ __forceinline__ double block_sum(double v, double* red) {
  const int t = threadIdx.x;
  red[t] = v;
  __syncthreads();
  for (int s = blockDim.x >> 1; s > 0; s >>= 1) {
    if (t < s) red[t] += red[t + s];
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  return r;
}

// Cholesky factors of the diagonal blocks of level columns c0..c1-1 (c1 - c0 <= 32 / D) by the 32
// lanes of one warp, in two parts.  diag_rows_factor: lane r of group g holds row r of column
// lvlcols[c0 + g]; step j shares the pivot row's entries by shuffles and updates the trailing
// rows (a right-looking column step per pivot); it stores L(k,k) and
// the reciprocal pivots (the diagonal of L(k,k)^-1).  diag_rows_inverse (after the stores are
// visible to the warp) reloads them and lane r computes column r of L(k,k)^-1.  All 32 lanes
// must call both (lanes beyond the last group work on an identity block and store nothing).
template <int D, class F>
__device__ __forceinline__ void diag_rows_factor(F& p, double* L, int c0, int c1, int* sflag, int gen) {
  constexpr int BS = D * D;
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int grp = lane / D, r = lane - grp * D, base = grp * D;
  const bool act = grp < c1 - c0;
  const int k = act ? p.lvlcols[c0 + grp] : 0;
  double* Lk = L + (int64_t)k * BS;
  double A[D], inv[D];
#pragma unroll
  for (int m = 0; m < D; ++m) A[m] = act ? Lk[r * D + m] : (m == r ? 1.0 : 0.0);
#pragma unroll
  for (int j = 0; j < D; ++j) {
    const double d = __shfl_sync(full, A[j], base + j);  // pivot A(j, j), already updated
    const double il = rsqrt(d);
    inv[j] = il;
    // L(j, j) = d / sqrt(d) on lane j, L(r, j) = A(r, j) / sqrt(d) below it; lanes above the
    // pivot row compute a value nobody reads
    const double lrj = (r == j ? d : A[j]) * il;
    A[j] = lrj;
#pragma unroll
    for (int m = j + 1; m < D; ++m) {
      const double lmj = __shfl_sync(full, lrj, base + m);
      A[m] = fma(-lrj, lmj, A[m]);  // entries right of the diagonal are never read or stored
    }
  }
  // a pivot that is not positive and finite leaves L(r, r) = d rsqrt(d) NaN (0 * inf, inf * 0
  // or the NaN of a negative square root), so one test of the row's own diagonal per lane
  // replaces a test per pivot
  const bool ok = A[r] > 0.0 && A[r] < INFINITY;
  if (act) {
#pragma unroll
    for (int m = 0; m < D; ++m) Lk[r * D + m] = m <= r ? A[m] : 0.0;
    p.Linv[(int64_t)k * BS + r * D + r] = inv[r];
    if (!ok) *sflag = gen;
  }
}

// Columns c0..c1-1 of `cols` (null: the columns c0..c1-1 themselves).
template <int D, class F>
__device__ __forceinline__ void diag_rows_inverse(F& p, const double* L, int c0, int c1,
                                                  const int32_t* cols) {
  constexpr int BS = D * D;
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int grp = lane / D, r = lane - grp * D, base = grp * D;
  const bool act = grp < c1 - c0;
  const int k = act ? (cols ? cols[c0 + grp] : c0 + grp) : 0;
  const double* Lk = L + (int64_t)k * BS;
  const double* Ik = p.Linv + (int64_t)k * BS;
  double A[D], inv[D];
#pragma unroll
  for (int m = 0; m < D; ++m) {
    A[m] = act ? Lk[r * D + m] : (m == r ? 1.0 : 0.0);
    inv[m] = act ? Ik[m * D + m] : 1.0;
  }
  // column r of L^-1: I(r, r) = 1 / L(r, r); I(i, r) = -(sum_{m=r}^{i-1} L(i, m) I(m, r)) / L(i, i)
  double I[D];
#pragma unroll
  for (int i = 0; i < D; ++i) I[i] = 0.0;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    if (i == r) I[i] = inv[i];
    double s = 0.0;
#pragma unroll
    for (int m = 0; m < i; ++m) {
      const double lim = __shfl_sync(full, A[m], base + i);  // L(i, m) from lane i
      if (m >= r) s += lim * I[m];
    }
    if (i > r) I[i] = -s * inv[i];
  }
  if (act) {
#pragma unroll
    for (int m = 0; m < D; ++m) p.Linv[(int64_t)k * BS + m * D + r] = I[m];
  }
}

// L(k,k)^-1 in FP32 from the FP32 factor copy Lf, into Linvf, for k = c0 .. c1-1, by the 32 lanes
// of one warp (lane r of group g: column r of block c0 + g, as diag_rows_inverse).  All 32 lanes
// must call it.
template <int D>
__device__ __forceinline__ void diag_rows_inverse_f32(const float* Lf, float* Linvf, int c0, int c1) {
  constexpr int BS = D * D;
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int grp = lane / D, r = lane - grp * D, base = grp * D;
  const bool act = grp < c1 - c0;
  const int k = act ? c0 + grp : 0;
  const float* Lk = Lf + (int64_t)k * BS;
  float A[D], I[D];
#pragma unroll
  for (int m = 0; m < D; ++m) A[m] = act ? Lk[r * D + m] : (m == r ? 1.0f : 0.0f);
#pragma unroll
  for (int i = 0; i < D; ++i) I[i] = 0.0f;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    const float lii = __shfl_sync(full, A[i], base + i);  // L(i, i) from lane i
    float s = 0.0f;
#pragma unroll
    for (int m = 0; m < i; ++m) {
      const float lim = __shfl_sync(full, A[m], base + i);  // L(i, m) from lane i
      if (m >= r) s += lim * I[m];
    }
    if (i == r) I[i] = 1.0f / lii;
    if (i > r) I[i] = -s / lii;
  }
  if (act) {
#pragma unroll
    for (int m = 0; m < D; ++m) Linvf[(int64_t)k * BS + m * D + r] = I[m];
  }
}

// Off-diagonal blocks of level lv's columns by forward substitution with L(k,k) and its
// reciprocal pivots (the diagonal of L(k,k)^-1, stored by diag_rows_factor):
// L(r,k) <- A(r,k) L(k,k)^-T, one row per thread of the team.
template <int D, class F>
__device__ __forceinline__ void panel_subst(F& p, double* L, int lv, int tid, int nthr) {
  constexpr int BS = D * D;
  const int q0 = p.panptr[lv], q1 = p.panptr[lv + 1];
  for (int it = tid; it < (q1 - q0) * D; it += nthr) {
    const int q = q0 + it / D, row = it % D;
    double* X = L + (int64_t)p.pan[2 * q] * BS + row * D;
    const int k = p.pan[2 * q + 1];
    const double* Lk = L + (int64_t)k * BS;
    const double* Ik = p.Linv + (int64_t)k * BS;
    double o[D];
#pragma unroll
    for (int jj = 0; jj < D; ++jj) {
      double s2 = X[jj];
#pragma unroll
      for (int mm = 0; mm < jj; ++mm) s2 = fma(-o[mm], Lk[jj * D + mm], s2);
      o[jj] = s2 * Ik[jj * D + jj];
    }
#pragma unroll
    for (int jj = 0; jj < D; ++jj) X[jj] = o[jj];
  }
}

// Subtracts from each target block t0 .. t1-1 (of the target list) the products of its source
// pairs: mode 0 all pairs, 1 the early ones (gptr .. gsplit), 2 the late ones (gsplit .. next
// gptr).  Each output element is summed by LN adjacent lanes (a power of two) and combined by a
// fixed-order shuffle reduction.  Runs on the team threads tid = 0 .. nthr-1 (whole warps: tid
// and nthr advance warp by warp, so every warp taking part is whole).
template <int D, class F>
__device__ __forceinline__ void gather_targets(F& p, double* L, int t0, int t1, int LN, int mode,
                                               int tid, int nthr) {
  constexpr int BS = D * D;
  const int lsh = __ffs(LN) - 1;
  const int n1 = (t1 - t0) * BS * LN;
  for (int base = 0; base < n1; base += nthr) {
    const int it = base + tid;
    double acc = 0.0;
    int q = 0, el = 0, s0 = 0, s1 = 0;
    if (it < n1) {
      const int e2 = it >> lsh, lane = it & (LN - 1);
      q = t0 + e2 / BS;
      el = e2 % BS;
      const int a = el / D, b = el % D;
      s0 = mode == 2 ? p.gsplit[q] : p.gptr[q];
      s1 = mode == 1 ? p.gsplit[q] : p.gptr[q + 1];
      for (int s = s0 + lane; s < s1; s += LN) {
        const double* X = L + (int64_t)p.gsrc[2 * s] * BS + a * D;
        const double* Y = L + (int64_t)p.gsrc[2 * s + 1] * BS + b * D;
#pragma unroll
        for (int mm = 0; mm < D; ++mm) acc = fma(X[mm], Y[mm], acc);
      }
    }
    if (LN > 1) acc = lane_sum(acc, LN);
    if (it < n1 && (it & (LN - 1)) == 0 && s1 > s0) L[(int64_t)p.tgt[q] * BS + el] -= acc;
  }
}

// The targets of level lv, LN = glanes[lv].
template <int D, class F>
__device__ __forceinline__ void gather_level(F& p, double* L, int lv, int mode, int tid, int nthr) {
  gather_targets<D>(p, L, p.tgtptr[lv], p.tgtptr[lv + 1], p.glanes[lv], mode, tid, nthr);
}

// L <- H (fill-in blocks zero) by the team threads tid = 0 .. nthr-1.  Each thread first fetches
// the source offsets of U elements, then the elements, then stores them, so its loads are in
// flight together.  damp_diagonal then adds lam * max(diag H, floor) + shift to the diagonal.
template <int D, class F>
__device__ __forceinline__ void load_factor(F& p, double* L, int tid, int nthr) {
  constexpr int BS = D * D, U = 4;
  const int total = (p.N + p.nnzL) * BS;
  for (int it0 = tid; it0 < total; it0 += U * nthr) {
    int off[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int it = it0 + u * nthr, t = it / BS, el = it - t * BS;
      int o = -1;
      if (it < total) {
        if (t < p.N) {
          o = it;
        } else {
          const int src = p.lsrc[t - p.N];
          o = src >= 0 ? (p.N + src) * BS + el : -1;
        }
      }
      off[u] = o;
    }
    double v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) v[u] = off[u] >= 0 ? p.H[off[u]] : 0.0;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int it = it0 + u * nthr;
      if (it < total) L[it] = v[u];
    }
  }
}

// The damping that follows load_factor (after a barrier), on the N * D diagonal entries.
template <int D, class F>
__device__ __forceinline__ void damp_diagonal(F& p, double* L, double lam, double shift, int tid,
                                              int nthr) {
  for (int it = tid; it < p.N * D; it += nthr) {
    const int t = it / D, a = it - t * D;
    double* x = L + (int64_t)t * D * D + a * (D + 1);
    *x += lam * fmax(*x, kDiagFloor) + shift;
  }
}

// Trailing update of dense-supernode column i (levels dense_lev .. nlev-1: one block column
// each, every block of the lower triangle stored): every block (r, s), i < s <= r, minus
// L(r,i) L(s,i)^T, one block row (D outputs, D^2 FMAs from registers) per item, items spread
// over the team threads tid = 0 .. nthr-1.
template <int D, class F>
__device__ __forceinline__ void supernode_trailing(F& p, double* L, int i, int tid, int nthr) {
  constexpr int BS = D * D;
  const int d0 = p.dense_lev, m = p.nlev - d0;
  const int M = m - 1 - i;  // trailing supernode columns
  // column i's off-diagonal blocks, rows i+1 .. m-1 of the supernode in order
  const double* P = L + (int64_t)(p.N + p.colptr[p.lvlcols[p.lvlptr[d0 + i]]]) * BS;
  // trailing blocks in column-major order: column s' (supernode column i+1+s') holds rows
  // r' = s' .. M-1 and starts at first(s') = s' M - s' (s' - 1) / 2.  T D fits in int32: the
  // whole factor of one problem is below 2^31 bytes.
  const int T = M * (M + 1) / 2;
  const int twoM1 = 2 * M + 1;
  for (int it = tid; it < T * D; it += nthr) {
    const int q = it / D, a = it - q * D;
    int sc = (int)(0.5f * ((float)twoM1 - sqrtf((float)(twoM1 * twoM1 - 8 * q))));
    sc = max(0, min(sc, M - 1));
    while (sc > 0 && sc * M - sc * (sc - 1) / 2 > q) --sc;
    while (sc + 1 < M && (sc + 1) * M - (sc + 1) * sc / 2 <= q) ++sc;
    const int rc = sc + q - (sc * M - sc * (sc - 1) / 2);
    const int ks = p.lvlcols[p.lvlptr[d0 + i + 1 + sc]];
    double* A = L + (int64_t)(rc == sc ? ks : p.N + p.colptr[ks] + (rc - sc - 1)) * BS + a * D;
    const double* Lr = P + (int64_t)rc * BS + a * D;
    const double* Ls = P + (int64_t)sc * BS;
    double x[D];
#pragma unroll
    for (int mm = 0; mm < D; ++mm) x[mm] = Lr[mm];
#pragma unroll
    for (int b = 0; b < D; ++b) {
      double acc = A[b];
#pragma unroll
      for (int mm = 0; mm < D; ++mm) acc = fma(-x[mm], Ls[b * D + mm], acc);
      A[b] = acc;
    }
  }
}

// supernode_trailing as a call with a register allocation of its own, for the cluster
// factorization: inlined into the cluster instance of the forward kernel, spill placement alone
// made its large-graph factorizations 2.2x slower (the single-CTA factorization keeps the inline
// form, whose allocation measured best there and which a call boundary would change for every
// problem size).
template <int D, class F>
__device__ __noinline__ void supernode_trailing_call(F& p, double* L, int i, int tid, int nthr) {
  supernode_trailing<D>(p, L, i, tid, nthr);
}

// The dense supernode, factored right-looking once the sparse levels are final: (1) every
// supernode block minus its products with sparse columns, one gather over all its targets;
// then for each supernode column i: (2) its diagonal block factored by warp 0, (3) its
// off-diagonal blocks L(r,i) by substitution, (4) the trailing update (supernode_trailing).
// The products are those of the level schedule, summed column by column.  Returns false
// (uniformly) on a pivot that is not positive and finite, after writing `gen` into *sflag.
template <int D, class F>
__device__ bool dense_supernode(F& p, double* L, int* sflag, int gen) {
  const int d0 = p.dense_lev, m = p.nlev - d0;
  gather_targets<D>(p, L, p.tgtptr[d0], p.tgtptr[p.nlev], p.glanes[p.nlev], 1, threadIdx.x,
                    blockDim.x);
  __syncthreads();
  for (int i = 0; i < m; ++i) {
    const int c0 = p.lvlptr[d0 + i];
    if (threadIdx.x < 32) diag_rows_factor<D>(p, L, c0, c0 + 1, sflag, gen);
    __syncthreads();
    if (*sflag == gen) return false;
    panel_subst<D>(p, L, d0 + i, threadIdx.x, blockDim.x);
    __syncthreads();
    if (m - 1 - i == 0) break;
    supernode_trailing<D>(p, L, i, threadIdx.x, blockDim.x);
    __syncthreads();
  }
  return true;
}

// L <- H + lam * diag(max(diag H, floor)) + shift * I, then left-looking block Cholesky level
// by level (the dense supernode, if any, right-looking after the sparse levels), and finally
// the inverses of the diagonal blocks (used by the solves only).
// Returns false (uniformly across the CTA) if a pivot is not positive or not finite.  A failing
// thread writes the call's generation number `gen` into *sflag; the flag is never reset, so a
// slow thread can never see a later call's state.
// inverse = false leaves out the final pass (L(k,k)^-1 then holds only its diagonal, the
// reciprocal pivots): for a caller that forms the inverses another way or later
// (diag_inverses).
template <int D, class F>
__device__ bool block_factor(F& p, double lam, int* sflag, int gen, double shift = 0.0,
                             bool inverse = true) {
  constexpr int CPW = 32 / D;  // diagonal blocks per warp in diag_rows_factor
  double* L = p.L;
  const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  load_factor<D>(p, L, threadIdx.x, blockDim.x);
  __syncthreads();
  damp_diagonal<D>(p, L, lam, shift, threadIdx.x, blockDim.x);
  __syncthreads();
  // Level by level: (1) gather, (2) diagonal factors, (3) panels.  On a narrow level (at most
  // CPW columns) warp 0 alone factors the diagonal blocks, and the other warps meanwhile
  // subtract the next level's "early" source pairs (columns two or more levels below, already
  // final); that level's gather then only adds the pairs from the level just factored.  On a
  // wide level every warp factors CPW diagonal blocks at a time.
  bool early_done = false;
  const int nsparse = p.dense_lev;  // levels of the level schedule
  for (int lv = 0; lv < nsparse; ++lv) {
    gather_level<D>(p, L, lv, early_done ? 2 : 0, threadIdx.x, blockDim.x);
    __syncthreads();
    const int c0 = p.lvlptr[lv], c1 = p.lvlptr[lv + 1];
    if (c1 - c0 <= CPW && nwarps >= 2) {
      if (warp == 0)
        diag_rows_factor<D>(p, L, c0, c1, sflag, gen);
      else if (lv + 1 < nsparse)
        gather_level<D>(p, L, lv + 1, 1, threadIdx.x - 32, blockDim.x - 32);
      early_done = lv + 1 < nsparse;
    } else {
      for (int cc = c0 + warp * CPW; cc < c1; cc += nwarps * CPW)
        diag_rows_factor<D>(p, L, cc, min(cc + CPW, c1), sflag, gen);
      early_done = false;
    }
    __syncthreads();
    if (*sflag == gen) return false;
    panel_subst<D>(p, L, lv, threadIdx.x, blockDim.x);
    __syncthreads();
  }
  if (nsparse < p.nlev && !dense_supernode<D>(p, L, sflag, gen)) return false;
  if (inverse) {
    for (int cc = warp * CPW; cc < p.N; cc += nwarps * CPW)
      diag_rows_inverse<D>(p, L, cc, min(cc + CPW, p.N), nullptr);
    __syncthreads();
  }
  return true;
}

// The inverse pass of block_factor on its own (after a factorization with inverse = false), by
// this CTA's warps.
template <int D, class F>
__device__ void diag_inverses(F& p) {
  constexpr int CPW = 32 / D;
  const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int cc = warp * CPW; cc < p.N; cc += nwarps * CPW)
    diag_rows_inverse<D>(p, p.L, cc, min(cc + CPW, p.N), nullptr);
  __syncthreads();
}

// ----------------------------------------------------------------------------- cluster factor

// block_factor by the nranks CTAs of a thread-block cluster (rank = the CTA's rank in it), for a
// factor too large for one SM's FP64 rate: the same level schedule and the same sums in the same
// order, with the gather, panel and wide-level items spread over all the cluster's threads, the
// narrow-level diagonal blocks factored by warp 0 of rank 0 while every other warp of the cluster
// takes the next level's early gather pairs, and cluster barriers between the phases; the dense
// supernode, if any, column by column as in dense_supernode with its gathers, panels and
// trailing updates spread the same way.  The factor lives in global memory; `gflag` (global, one
// per problem, set to -1 before the first call of a launch and published by a cluster barrier)
// records a failed pivot as for block_factor.  Returns the same value in every thread of the
// cluster, right after a cluster barrier.  kDense = false compiles the supernode part out (for
// structures analysed without one).
template <int D, bool kDense = true, class F>
__device__ bool block_factor_cluster(F& p, double lam, int rank, int nranks, int* gflag, int gen,
                                     double shift = 0.0, bool inverse = true) {
  double* L = p.L;
  // team index: consecutive warps of work go to consecutive CTAs, so that a phase with fewer
  // items than the cluster has threads still spreads over all of the cluster's SMs
  const int tid = ((threadIdx.x >> 5) * nranks + rank) * 32 + (threadIdx.x & 31);
  const int nthr = nranks * blockDim.x;
  load_factor<D>(p, L, tid, nthr);
  cluster_sync_all();
  damp_diagonal<D>(p, L, lam, shift, tid, nthr);
  cluster_sync_all();
  constexpr int CPW = 32 / D;  // diagonal blocks per warp in diag_rows_factor
  const int warp = tid >> 5, nwarps = nthr >> 5;
  const int nsparse = kDense ? p.dense_lev : p.nlev;  // levels of the level schedule
  bool early_done = false;
  for (int lv = 0; lv < nsparse; ++lv) {
    gather_level<D>(p, L, lv, early_done ? 2 : 0, tid, nthr);
    cluster_sync_all();
    const int c0 = p.lvlptr[lv], c1 = p.lvlptr[lv + 1];
    if (c1 - c0 <= CPW) {
      if (warp == 0)
        diag_rows_factor<D>(p, L, c0, c1, gflag, gen);
      else if (lv + 1 < nsparse)
        gather_level<D>(p, L, lv + 1, 1, tid - 32, nthr - 32);
      early_done = lv + 1 < nsparse;
    } else {
      for (int cc = c0 + warp * CPW; cc < c1; cc += nwarps * CPW)
        diag_rows_factor<D>(p, L, cc, min(cc + CPW, c1), gflag, gen);
      early_done = false;
    }
    cluster_sync_all();
    if (*(volatile int*)gflag == gen) return false;
    panel_subst<D>(p, L, lv, tid, nthr);
    cluster_sync_all();
  }
  if (kDense && nsparse < p.nlev) {
    const int m = p.nlev - nsparse;
    gather_targets<D>(p, L, p.tgtptr[nsparse], p.tgtptr[p.nlev], p.glanes[p.nlev], 1, tid, nthr);
    cluster_sync_all();
    for (int i = 0; i < m; ++i) {
      const int c0 = p.lvlptr[nsparse + i];
      if (warp == 0) diag_rows_factor<D>(p, L, c0, c0 + 1, gflag, gen);
      cluster_sync_all();
      if (*(volatile int*)gflag == gen) return false;
      panel_subst<D>(p, L, nsparse + i, tid, nthr);
      cluster_sync_all();
      if (m - 1 - i == 0) break;
      supernode_trailing_call<D>(p, L, i, tid, nthr);
      cluster_sync_all();
    }
  }
  if (inverse) {
    for (int cc = warp * CPW; cc < p.N; cc += nwarps * CPW)
      diag_rows_inverse<D>(p, L, cc, min(cc + CPW, p.N), nullptr);
    cluster_sync_all();
  }
  return true;
}

// In place: x <- (L L^T)^-1 x (positions order, FP64), level by level.  kTopChain = false leaves
// out the top chain's pre-pass (the same result up to summation order, less code: used where
// registers are scarce).
// Forward and back substitution with the block factor, in the scalar type T of the given
// factor copy (L, Linv: blocks as in p.L / p.Linv) and vectors (x: right-hand side in, solution
// out; tmp: scratch of the same length).
template <int D, bool kTopChain, class T, class F>
__device__ void block_solve_t(F& p, const T* L, const T* Linv, T* x, T* tmp) {
  const int chain_lev = kTopChain ? p.chain_lev : p.nlev;
  constexpr int BS = D * D;
  for (int lv = 0; lv < p.nlev; ++lv) {
    const int c0 = p.lvlptr[lv], c1 = p.lvlptr[lv + 1];
    // Rows of the top chain (levels chain_lev.., one column each): their pairs from columns
    // outside the chain, whose values are final once the levels below are done, are summed for
    // all chain rows at once before the first chain level; each chain level then only adds the
    // pairs from chain columns (rowent from rsplit[k] on).
    const bool chain = lv >= chain_lev;
    if (lv == chain_lev) {
      const int LN = p.slanes[p.nlev], lsh = __ffs(LN) - 1;
      const int n1 = (p.nlev - lv) * D * LN;
      for (int base = 0; base < n1; base += blockDim.x) {
        const int it = base + threadIdx.x;
        T acc = T(0);
        int k = 0, i = 0;
        if (it < n1) {
          const int e2 = it >> lsh, lane = it & (LN - 1);
          k = p.lvlcols[c0 + e2 / D];
          i = e2 % D;
          for (int q = p.rowptr[k] + lane; q < p.rsplit[k]; q += LN) {
            const T* B = L + (int64_t)p.rowent[2 * q] * BS + i * D;
            const T* y = x + p.rowent[2 * q + 1] * D;
#pragma unroll
            for (int mm = 0; mm < D; ++mm) acc = fma_t(B[mm], y[mm], acc);
          }
        }
        if (LN > 1) acc = lane_sum(acc, LN);
        if (it < n1 && (it & (LN - 1)) == 0) tmp[k * D + i] = x[k * D + i] - acc;
      }
      __syncthreads();
    }
    const int LN = p.slanes[lv], lsh = __ffs(LN) - 1;  // LN is a power of two
    const int n1 = (c1 - c0) * D * LN;
    for (int base = 0; base < n1; base += blockDim.x) {
      const int it = base + threadIdx.x;
      T acc = T(0);
      int k = 0, i = 0;
      if (it < n1) {
        const int e2 = it >> lsh, lane = it & (LN - 1);
        k = p.lvlcols[c0 + e2 / D];
        i = e2 % D;
        for (int q = (chain ? p.rsplit[k] : p.rowptr[k]) + lane; q < p.rowptr[k + 1]; q += LN) {
          const T* B = L + (int64_t)p.rowent[2 * q] * BS + i * D;
          const T* y = x + p.rowent[2 * q + 1] * D;
#pragma unroll
          for (int mm = 0; mm < D; ++mm) acc = fma_t(B[mm], y[mm], acc);
        }
      }
      if (LN > 1) acc = lane_sum(acc, LN);
      if (it < n1 && (it & (LN - 1)) == 0) tmp[k * D + i] = (chain ? tmp[k * D + i] : x[k * D + i]) - acc;
    }
    __syncthreads();
    for (int it = threadIdx.x; it < (c1 - c0) * D; it += blockDim.x) {
      const int k = p.lvlcols[c0 + it / D], i = it % D;
      const T* I = Linv + (int64_t)k * BS + i * D;
      T s = T(0);
#pragma unroll
      for (int mm = 0; mm < D; ++mm)
        if (mm <= i) s = fma_t(I[mm], tmp[k * D + mm], s);
      x[k * D + i] = s;
    }
    __syncthreads();
  }
  for (int lv = p.nlev - 1; lv >= 0; --lv) {
    const int c0 = p.lvlptr[lv], c1 = p.lvlptr[lv + 1];
    const int LN = p.slanes[lv], lsh = __ffs(LN) - 1;  // LN is a power of two
    const int n1 = (c1 - c0) * D * LN;
    for (int base = 0; base < n1; base += blockDim.x) {
      const int it = base + threadIdx.x;
      T acc = T(0);
      int k = 0, i = 0;
      if (it < n1) {
        const int e2 = it >> lsh, lane = it & (LN - 1);
        k = p.lvlcols[c0 + e2 / D];
        i = e2 % D;
        const int basec = p.colptr[k];
        const int cnt = p.colptr[k + 1] - basec;
        for (int aa = lane; aa < cnt; aa += LN) {
          const T* B = L + (int64_t)(p.N + basec + aa) * BS + i;
          const T* y = x + p.rows[basec + aa] * D;
#pragma unroll
          for (int mm = 0; mm < D; ++mm) acc = fma_t(B[mm * D], y[mm], acc);
        }
      }
      if (LN > 1) acc = lane_sum(acc, LN);
      if (it < n1 && (it & (LN - 1)) == 0) tmp[k * D + i] = x[k * D + i] - acc;
    }
    __syncthreads();
    for (int it = threadIdx.x; it < (c1 - c0) * D; it += blockDim.x) {
      const int k = p.lvlcols[c0 + it / D], i = it % D;
      const T* I = Linv + (int64_t)k * BS;
      T s = T(0);
#pragma unroll
      for (int mm = 0; mm < D; ++mm)
        if (mm >= i) s = fma_t(I[mm * D + i], tmp[k * D + mm], s);
      x[k * D + i] = s;
    }
    __syncthreads();
  }
}

template <int D, bool kTopChain = true, class F>
__device__ void block_solve(F& p, double* x) {
  block_solve_t<D, kTopChain, double>(p, p.L, p.Linv, x, p.tmp);
}


}  // namespace dnls
