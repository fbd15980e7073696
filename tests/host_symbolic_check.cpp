// Host-side check of the symbolic analysis (no GPU): reads graphs from stdin, runs
// build_graph_host, and verifies the invariants the CUDA factorization and solves rely on.
// Input: B, then per problem "N E" and E lines "i j" (j = -1 for a prior).
// Output: one line per problem "ok <nlev> <chain_lev> <flops> <dense_lev> <residual>" or
// "fail <reason>" (the residual: of the host emulation of the device factorization).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <random>
#include <set>
#include <vector>

#include "dnls.h"
#include "../paper_2207_09442_b300/csrc/dnls_graph.h"

using namespace dnls;

static bool pow2_le8(int v) { return v == 1 || v == 2 || v == 4 || v == 8; }

// The factorization the CUDA kernels run, written as plain loops over the symbolic structure
// (any out-of-range index returns a residual of 1e30).  Returns max |L L^T - A| / max |A| over
// sampled rows.
static double emulate(const ProbMeta& m, const int32_t* s, int64_t Nl, const int32_t* ei,
                      const int32_t* ej, int E) {
  constexpr int D = 6, BS = 36;
  const int N = (int)Nl, nnzL = m.nnzL, nlev = m.nlev, dl = m.dense_lev;
  const int32_t *iperm = s + m.o_iperm, *colptr = s + m.o_colptr, *rows = s + m.o_rows,
                *lvlptr = s + m.o_lvlptr, *lvlcols = s + m.o_lvlcols, *tgtptr = s + m.o_tgtptr,
                *tgt = s + m.o_tgt, *gptr = s + m.o_gptr, *gsrc = s + m.o_gsrc,
                *gsplit = s + m.o_gsplit, *panptr = s + m.o_panptr, *pan = s + m.o_pan;
  const int NB = N + nnzL, nd = N * D;
  std::vector<double> A((size_t)nd * nd, 0.0);
  std::mt19937_64 rng(12345 + N);
  std::normal_distribution<double> nrm;
  for (int e = 0; e < E; ++e) {
    const int pi = iperm[ei[e]], pj = ej[e] >= 0 ? iperm[ej[e]] : -1;
    double Bm[6][12];
    for (auto& r : Bm)
      for (double& x : r) x = nrm(rng);
    int idx[12];
    for (int a = 0; a < 6; ++a) {
      idx[a] = pi * D + a;
      idx[6 + a] = pj >= 0 ? pj * D + a : -1;
    }
    for (int u = 0; u < 12; ++u)
      for (int v = 0; v < 12; ++v) {
        if (idx[u] < 0 || idx[v] < 0) continue;
        double acc = 0;
        for (int k = 0; k < 6; ++k) acc += Bm[k][u] * Bm[k][v];
        A[(size_t)idx[u] * nd + idx[v]] += acc;
      }
  }
  for (int i = 0; i < nd; ++i) A[(size_t)i * nd + i] += 1.0;
  std::vector<double> L((size_t)NB * BS, 0.0);
  for (int c = 0; c < N; ++c) {
    for (int x = 0; x < D; ++x)
      for (int y = 0; y < D; ++y) L[(size_t)c * BS + x * D + y] = A[(size_t)(c * D + x) * nd + c * D + y];
    for (int a = colptr[c]; a < colptr[c + 1]; ++a)
      for (int x = 0; x < D; ++x)
        for (int y = 0; y < D; ++y)
          L[(size_t)(N + a) * BS + x * D + y] = A[(size_t)(rows[a] * D + x) * nd + c * D + y];
  }
  bool bad = false;
  auto inb = [&](int64_t id) { if (id < 0 || id >= NB) bad = true; return !bad; };
  auto gather = [&](int t0, int t1, bool early_only) {
    for (int q = t0; q < t1 && !bad; ++q) {
      const int s0 = gptr[q], s1 = early_only ? gsplit[q] : gptr[q + 1];
      if (!inb(tgt[q])) return;
      for (int el = 0; el < BS; ++el) {
        const int a = el / D, bb = el % D;
        double acc = 0;
        for (int pq = s0; pq < s1; ++pq) {
          if (!inb(gsrc[2 * pq]) || !inb(gsrc[2 * pq + 1])) return;
          for (int mm = 0; mm < D; ++mm)
            acc += L[(size_t)gsrc[2 * pq] * BS + a * D + mm] * L[(size_t)gsrc[2 * pq + 1] * BS + bb * D + mm];
        }
        L[(size_t)tgt[q] * BS + el] -= acc;
      }
    }
  };
  auto diag = [&](int k) {
    double* Lk = &L[(size_t)k * BS];
    for (int j = 0; j < D; ++j) {
      const double d = Lk[j * D + j];
      if (!(d > 0)) { bad = true; return; }
      const double sq = std::sqrt(d);
      Lk[j * D + j] = sq;
      for (int r = j + 1; r < D; ++r) Lk[r * D + j] /= sq;
      for (int r = j + 1; r < D; ++r)
        for (int c = j + 1; c <= r; ++c) Lk[r * D + c] -= Lk[r * D + j] * Lk[c * D + j];
    }
    for (int r = 0; r < D; ++r)
      for (int c = r + 1; c < D; ++c) Lk[r * D + c] = 0;
  };
  auto panel = [&](int lv) {
    for (int q = panptr[lv]; q < panptr[lv + 1] && !bad; ++q) {
      if (!inb(pan[2 * q]) || pan[2 * q + 1] < 0 || pan[2 * q + 1] >= N) { bad = true; return; }
      double* X = &L[(size_t)pan[2 * q] * BS];
      const double* Lk = &L[(size_t)pan[2 * q + 1] * BS];
      for (int row = 0; row < D; ++row)
        for (int jj = 0; jj < D; ++jj) {
          double s2 = X[row * D + jj];
          for (int mm = 0; mm < jj; ++mm) s2 -= X[row * D + mm] * Lk[jj * D + mm];
          X[row * D + jj] = s2 / Lk[jj * D + jj];
        }
    }
  };
  for (int lv = 0; lv < dl && !bad; ++lv) {
    gather(tgtptr[lv], tgtptr[lv + 1], false);
    for (int c = lvlptr[lv]; c < lvlptr[lv + 1] && !bad; ++c) diag(lvlcols[c]);
    panel(lv);
  }
  if (dl < nlev && !bad) {
    gather(tgtptr[dl], tgtptr[nlev], true);
    const int mc = nlev - dl;
    for (int i = 0; i < mc && !bad; ++i) {
      const int c0 = lvlptr[dl + i];
      diag(lvlcols[c0]);
      panel(dl + i);
      const int M = mc - 1 - i;
      if (M == 0 || bad) break;
      const int ki = lvlcols[c0];
      const size_t P = (size_t)(N + colptr[ki]) * BS;
      const int T = M * (M + 1) / 2, twoM1 = 2 * M + 1;
      for (int it = 0; it < T * D && !bad; ++it) {  // every thread's item, mapped as the kernel does
        const int q = it / D, a = it - q * D;
        int sc = (int)(0.5f * ((float)twoM1 - std::sqrt((float)(twoM1 * twoM1 - 8 * q))));
        sc = std::max(0, std::min(sc, M - 1));
        while (sc > 0 && sc * M - sc * (sc - 1) / 2 > q) --sc;
        while (sc + 1 < M && (sc + 1) * M - (sc + 1) * sc / 2 <= q) ++sc;
        const int rc = sc + q - (sc * M - sc * (sc - 1) / 2);
        if (rc < sc || rc >= M) { bad = true; break; }
        const int ks = lvlcols[lvlptr[dl + i + 1 + sc]];
        const int64_t tb = rc == sc ? ks : N + colptr[ks] + (rc - sc - 1);
        if (!inb(tb)) break;
        double* Ab = &L[(size_t)tb * BS + a * D];
        for (int bb = 0; bb < D; ++bb) {
          double acc = Ab[bb];
          for (int mm = 0; mm < D; ++mm)
            acc -= L[P + (size_t)rc * BS + a * D + mm] * L[P + (size_t)sc * BS + bb * D + mm];
          Ab[bb] = acc;
        }
      }
    }
  }
  if (bad) return 1e30;
  // L L^T against A on sampled rows
  std::vector<double> Ld((size_t)nd * nd, 0.0);
  for (int c = 0; c < N; ++c) {
    for (int x = 0; x < D; ++x)
      for (int y = 0; y < D; ++y) Ld[(size_t)(c * D + x) * nd + c * D + y] = L[(size_t)c * BS + x * D + y];
    for (int a = colptr[c]; a < colptr[c + 1]; ++a)
      for (int x = 0; x < D; ++x)
        for (int y = 0; y < D; ++y)
          Ld[(size_t)(rows[a] * D + x) * nd + c * D + y] = L[(size_t)(N + a) * BS + x * D + y];
  }
  double err = 0, mx = 0;
  const int stride = std::max(1, nd / 48);
  for (int i = 0; i < nd; i += stride)
    for (int j = 0; j <= i; ++j) {
      double acc = 0;
      for (int k = 0; k <= j; ++k) acc += Ld[(size_t)i * nd + k] * Ld[(size_t)j * nd + k];
      err = std::max(err, std::fabs(acc - A[(size_t)i * nd + j]));
      mx = std::max(mx, std::fabs(A[(size_t)i * nd + j]));
    }
  return err / mx;
}

int main() {
  int B = 0;
  if (scanf("%d", &B) != 1 || B < 1) return 2;
  std::vector<int64_t> po{0}, eo{0};
  std::vector<int32_t> ei, ej;
  for (int b = 0; b < B; ++b) {
    int n = 0, e = 0;
    if (scanf("%d %d", &n, &e) != 2) return 2;
    po.push_back(po.back() + n);
    eo.push_back(eo.back() + e);
    for (int k = 0; k < e; ++k) {
      int a = 0, c = 0;
      if (scanf("%d %d", &a, &c) != 2) return 2;
      ei.push_back(a);
      ej.push_back(c);
    }
  }
  GraphHost G;
  const int rc = build_graph_host(DNLS_SE3, B, po.data(), eo.data(), ei.data(), ej.data(),
                                  DNLS_ORDER_MIN_DEGREE, &G);
  if (rc != 0) {
    printf("fail build %d\n", rc);
    return 0;
  }
  for (int b = 0; b < B; ++b) {
    const ProbMeta& m = G.meta[b];
    const int32_t* s = G.sym.data() + m.sym;
    const int N = m.N, nlev = m.nlev;
    const int32_t *colptr = s + m.o_colptr, *rows = s + m.o_rows, *rowptr = s + m.o_rowptr,
                  *rowent = s + m.o_rowent, *rsplit = s + m.o_rsplit, *lvlptr = s + m.o_lvlptr,
                  *lvlcols = s + m.o_lvlcols, *tgtptr = s + m.o_tgtptr, *tgt = s + m.o_tgt,
                  *gptr = s + m.o_gptr, *gsrc = s + m.o_gsrc, *gsplit = s + m.o_gsplit,
                  *glanes = s + m.o_glanes, *slanes = s + m.o_slanes, *lsrc = s + m.o_lsrc,
                  *pairtgt = s + m.o_pairtgt, *perm = s + m.o_perm, *iperm = s + m.o_iperm;
    auto fail = [&](const char* why) { printf("fail %d %s\n", b, why); };
    // permutation
    bool ok = true;
    for (int k = 0; k < N && ok; ++k) ok = perm[k] >= 0 && perm[k] < N && iperm[perm[k]] == k;
    if (!ok) { fail("perm"); continue; }
    // levels: every column once; a column's first off-diagonal row (its parent) sits on a
    // higher level
    std::vector<int> lev(N, -1);
    for (int l = 0; l < nlev; ++l)
      for (int c = lvlptr[l]; c < lvlptr[l + 1]; ++c) {
        if (lev[lvlcols[c]] != -1) ok = false;
        lev[lvlcols[c]] = l;
      }
    for (int k = 0; k < N && ok; ++k) {
      ok = lev[k] >= 0;
      for (int a = colptr[k]; a < colptr[k + 1] && ok; ++a)
        ok = rows[a] > k && lev[rows[a]] > lev[k] && (a == colptr[k] || rows[a] > rows[a - 1]);
    }
    if (!ok) { fail("levels"); continue; }
    // top chain: the levels from chain_lev on hold one column each, the level below it more
    if (m.chain_lev < 0 || m.chain_lev > nlev) { fail("chain_lev range"); continue; }
    for (int l = m.chain_lev; l < nlev && ok; ++l) ok = lvlptr[l + 1] - lvlptr[l] == 1;
    if (ok && m.chain_lev < nlev && m.chain_lev > 0) ok = lvlptr[m.chain_lev] - lvlptr[m.chain_lev - 1] > 1;
    if (ok && m.chain_lev < nlev) ok = nlev - m.chain_lev >= 2;
    if (!ok) { fail("chain"); continue; }
    // rows: entries (block, column) with the columns outside the chain before rsplit[k]
    for (int k = 0; k < N && ok; ++k) {
      ok = rsplit[k] >= rowptr[k] && rsplit[k] <= rowptr[k + 1];
      for (int q = rowptr[k]; q < rowptr[k + 1] && ok; ++q) {
        const int blk = rowent[2 * q], j = rowent[2 * q + 1];
        const bool in_chain = lev[j] >= m.chain_lev;
        ok = j < k && blk >= N && blk < N + m.nnzL && (in_chain == (q >= rsplit[k])) &&
             (lev[k] >= m.chain_lev || !in_chain);
        // the block id must be L(k, j): row k in column j's structure
        if (ok) ok = rows[blk - N] == k && blk - N >= colptr[j] && blk - N < colptr[j + 1];
      }
    }
    if (!ok) { fail("rows"); continue; }
    // lanes: powers of two up to 8, one per level plus the chain pre-pass
    for (int l = 0; l < nlev && ok; ++l) ok = pow2_le8(glanes[l]) && pow2_le8(slanes[l]);
    if (ok) ok = pow2_le8(slanes[nlev]);
    if (!ok) { fail("lanes"); continue; }
    // dense supernode: levels dense_lev .. nlev-1 are top-chain levels whose columns hold every
    // chain column above them as rows (explicit zeros included)
    const int dl = m.dense_lev;
    if (dl < 0 || dl > nlev || (dl < nlev && dl != m.chain_lev)) { fail("dense_lev"); continue; }
    for (int l = dl; l < nlev && ok; ++l) {
      const int k = lvlcols[lvlptr[l]];
      ok = colptr[k + 1] - colptr[k] == nlev - 1 - l;
      for (int a = colptr[k]; a < colptr[k + 1] && ok; ++a)
        ok = rows[a] == lvlcols[lvlptr[l + 1 + (a - colptr[k])]];
    }
    if (ok) ok = pow2_le8(glanes[nlev]);
    if (!ok) { fail("supernode"); continue; }
    // gather lists: each target of level l is a block of one of its columns, source pairs
    // come from columns on lower levels, the early pairs (levels <= l - 2) first; targets in
    // a level are ordered by non-increasing pair count.  In the supernode the lists hold only
    // the pairs from sparse columns, all early.  The pair count matches the structure: column j
    // of a sparse level with c_j off-diagonal blocks gives c_j (c_j + 1) / 2 pairs.
    int64_t want_pairs = 0;
    for (int j = 0; j < N; ++j)
      if (lev[j] < dl) {
        const int64_t c = colptr[j + 1] - colptr[j];
        want_pairs += c * (c + 1) / 2;
      }
    int64_t pairs = 0;
    for (int l = 0; l < nlev && ok; ++l)
      for (int t = tgtptr[l]; t < tgtptr[l + 1] && ok; ++t) {
        const int target = tgt[t];
        int col = target < N ? target : -1;
        if (target >= N)
          for (int k = 0; k < N; ++k)
            if (target - N >= colptr[k] && target - N < colptr[k + 1]) col = k;
        ok = col >= 0 && lev[col] == l && gsplit[t] >= gptr[t] && gsplit[t] <= gptr[t + 1] &&
             gptr[t + 1] > gptr[t];
        if (ok && t > tgtptr[l]) ok = gptr[t + 1] - gptr[t] <= gptr[t] - gptr[t - 1];
        for (int q = gptr[t]; q < gptr[t + 1] && ok; ++q) {
          const int x = gsrc[2 * q], y = gsrc[2 * q + 1];
          ok = x >= N && y >= N && x < N + m.nnzL && y < N + m.nnzL;
          int jx = -1;
          for (int k = 0; k < N && ok; ++k)
            if (x - N >= colptr[k] && x - N < colptr[k + 1]) jx = k;
          if (l < dl)
            ok = ok && jx >= 0 && lev[jx] < l && ((lev[jx] <= l - 2) == (q < gsplit[t]));
          else
            ok = ok && jx >= 0 && lev[jx] < dl && q < gsplit[t];
        }
        pairs += gptr[t + 1] - gptr[t];
      }
    if (ok) ok = pairs == want_pairs;
    if (!ok) { fail("gather"); continue; }
    // assembly map: every pose pair's L block, and lsrc its inverse
    std::set<int> seen;
    for (int p = 0; p < m.npair && ok; ++p) {
      ok = pairtgt[p] >= N && pairtgt[p] < N + m.nnzL && lsrc[pairtgt[p] - N] == p;
      seen.insert(pairtgt[p]);
    }
    for (int t = 0; t < m.nnzL && ok; ++t) ok = (lsrc[t] >= 0) == (seen.count(N + t) > 0);
    if (!ok) { fail("assembly map"); continue; }
    // numeric emulation of the device factorization on A = sum over costs of B^T B + I (B a
    // seeded random 6 x 12 on the cost's two poses, the graph's sparsity): the level schedule's
    // gathers, diagonal factors and panels, then the supernode's gather of its sparse sources
    // and its right-looking trailing updates with the kernel's block-row mapping (the
    // column-major triangle index inverted through a float square root); L L^T against A.
    const double resid = emulate(m, s, po[b + 1] - po[b], ei.data() + eo[b], ej.data() + eo[b],
                                 (int)(eo[b + 1] - eo[b]));
    if (!(resid < 1e-12)) { fail("emulated factor"); continue; }
    printf("ok %d %d %.0f %d %.3g\n", nlev, m.chain_lev, G.prob_flops[b], dl, resid);
  }
  return 0;
}
