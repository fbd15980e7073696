// Host-side check of the symbolic analysis (no GPU): reads graphs from stdin, runs
// build_graph_host, and verifies the invariants the CUDA factorization and solves rely on.
// Input: B, then per problem "N E" and E lines "i j" (j = -1 for a prior).
// Output: one line per problem "ok <nlev> <chain_lev> <flops>" or "fail <reason>".
#include <cstdio>
#include <cstdlib>
#include <set>
#include <vector>

#include "dnls.h"
#include "../paper_2207_09442_b300/csrc/dnls_graph.h"

using namespace dnls;

static bool pow2_le8(int v) { return v == 1 || v == 2 || v == 4 || v == 8; }

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
    // gather lists: each target of level l is a block of one of its columns, source pairs
    // come from columns on lower levels, the early pairs (levels <= l - 2) first; targets in
    // a level are ordered by non-increasing pair count; the update count matches n_upd
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
          ok = ok && jx >= 0 && lev[jx] < l && ((lev[jx] <= l - 2) == (q < gsplit[t]));
        }
        pairs += gptr[t + 1] - gptr[t];
      }
    if (ok) ok = pairs == m.n_upd;
    if (!ok) { fail("gather"); continue; }
    // assembly map: every pose pair's L block, and lsrc its inverse
    std::set<int> seen;
    for (int p = 0; p < m.npair && ok; ++p) {
      ok = pairtgt[p] >= N && pairtgt[p] < N + m.nnzL && lsrc[pairtgt[p] - N] == p;
      seen.insert(pairtgt[p]);
    }
    for (int t = 0; t < m.nnzL && ok; ++t) ok = (lsrc[t] >= 0) == (seen.count(N + t) > 0);
    if (!ok) { fail("assembly map"); continue; }
    printf("ok %d %d %.0f\n", nlev, m.chain_lev, G.prob_flops[b]);
  }
  return 0;
}
