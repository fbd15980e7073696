// Host-side symbolic analysis of a batch of pose graphs (done once per structure and reused by
// every numeric factorization, as the paper's sparse solvers do, Sec. 4.2 and App. E):
//   1. a fill-reducing ordering of the pose blocks (minimum degree on the pose graph, ties to
//      the lowest index; or the natural order);
//   2. the block structure of the Cholesky factor L by symbolic elimination;
//   3. the elimination-tree level of every block column (a column depends only on its
//      descendants, so all columns of one level can be factored concurrently);
//   4. for every block of L, the list of (L(r,j), L(k,j)) products a left-looking
//      factorization subtracts from it, so that each block is reduced by one thread group in a
//      fixed order (no atomics, bitwise reproducible);
//   5. the assembly maps from costs to the blocks of H and the workspace plan.
#include <algorithm>
#include <cstring>
#include <map>

#include "../../include/dnls.h"
#include "dnls_graph.h"

namespace dnls {

namespace {

struct Bits {
  int words = 0;
  std::vector<uint64_t> w;
  void init(int n) { words = (n + 63) / 64; w.assign((size_t)words, 0); }
  void set(int i) { w[i >> 6] |= (uint64_t)1 << (i & 63); }
  void clr(int i) { w[i >> 6] &= ~((uint64_t)1 << (i & 63)); }
  bool get(int i) const { return (w[i >> 6] >> (i & 63)) & 1; }
};

int popcount_and(const Bits& a, const Bits& b) {
  int c = 0;
  for (int k = 0; k < a.words; ++k) c += __builtin_popcountll(a.w[k] & b.w[k]);
  return c;
}

// Eliminates the pose graph in the chosen order; returns the elimination order (position ->
// pose) and, per position, the poses adjacent at elimination time (the column structure).
void eliminate(int N, const std::vector<std::vector<int>>& adj0, bool min_degree,
               std::vector<int>& order, std::vector<std::vector<int>>& struct_poses) {
  std::vector<Bits> adj(N);
  for (int v = 0; v < N; ++v) {
    adj[v].init(N);
    for (int u : adj0[v]) adj[v].set(u);
  }
  Bits alive;
  alive.init(N);
  for (int v = 0; v < N; ++v) alive.set(v);
  std::vector<int> deg(N);
  for (int v = 0; v < N; ++v) deg[v] = (int)adj0[v].size();
  order.clear();
  struct_poses.assign(N, {});
  for (int step = 0; step < N; ++step) {
    int k = -1;
    if (min_degree) {
      int best = 1 << 30;
      for (int v = 0; v < N; ++v)
        if (alive.get(v) && deg[v] < best) { best = deg[v]; k = v; }
    } else {
      k = step;
    }
    order.push_back(k);
    alive.clr(k);
    std::vector<int> nb;
    for (int wd = 0; wd < adj[k].words; ++wd) {
      uint64_t m = adj[k].w[wd] & alive.w[wd];
      while (m) {
        int bit = __builtin_ctzll(m);
        nb.push_back(wd * 64 + bit);
        m &= m - 1;
      }
    }
    struct_poses[step] = nb;
    for (int x : nb) {
      for (int wd = 0; wd < adj[x].words; ++wd) adj[x].w[wd] |= adj[k].w[wd] & alive.w[wd];
      adj[x].clr(x);
      adj[x].clr(k);
    }
    for (int x : nb) deg[x] = popcount_and(adj[x], alive);
  }
}

int64_t align256(int64_t x) { return (x + 255) & ~(int64_t)255; }

}  // namespace

int build_graph_host(int kind, int B, const int64_t* pose_offsets, const int64_t* edge_offsets,
                     const int32_t* edge_i, const int32_t* edge_j, int ordering, GraphHost* out,
                     int threads, bool dense_chain) {
  if (!out || !pose_offsets || !edge_offsets || !edge_i || !edge_j) return DNLS_ERR_ARG;
  if ((kind != DNLS_SE2 && kind != DNLS_SE3) || B < 1) return DNLS_ERR_ARG;
  if (ordering != DNLS_ORDER_MIN_DEGREE && ordering != DNLS_ORDER_NATURAL) return DNLS_ERR_ARG;
  if (pose_offsets[0] != 0 || edge_offsets[0] != 0) return DNLS_ERR_ARG;
  GraphHost& G = *out;
  G.kind = kind;
  G.dof = kind == DNLS_SE3 ? 6 : 3;
  G.pw = kind == DNLS_SE3 ? 12 : 4;
  G.B = B;
  G.P_total = pose_offsets[B];
  G.E_total = edge_offsets[B];
  const int D = G.dof, BS = D * D;
  G.meta.assign(B, ProbMeta{});
  G.sym.clear();
  G.ei.assign(edge_i, edge_i + G.E_total);
  G.ej.assign(edge_j, edge_j + G.E_total);
  G.max_L_bytes = 0;
  G.max_nlev = 0;
  G.max_arena_bytes = 0;
  G.n_blocks_L = 0;
  G.n_upd = 0;
  G.factor_flops = 0;
  G.dense_flops = 0;
  int64_t ws = kWsHeader;
  int64_t dense_off = 0;
  std::vector<double> cost(B);

  for (int b = 0; b < B; ++b) {
    const int64_t p0 = pose_offsets[b], p1 = pose_offsets[b + 1];
    const int64_t e0 = edge_offsets[b], e1 = edge_offsets[b + 1];
    if (p1 <= p0 || e1 < e0) return DNLS_ERR_ARG;
    if (p1 - p0 > (1 << 20) || e1 - e0 > (1 << 24)) return DNLS_ERR_ARG;
    const int N = (int)(p1 - p0), E = (int)(e1 - e0);
    std::vector<std::vector<int>> adj(N);
    for (int e = 0; e < E; ++e) {
      int i = edge_i[e0 + e], j = edge_j[e0 + e];
      if (i < 0 || i >= N || j < -1 || j >= N || j == i) return DNLS_ERR_ARG;
      if (j >= 0) {
        adj[i].push_back(j);
        adj[j].push_back(i);
      }
    }
    for (auto& a : adj) {
      std::sort(a.begin(), a.end());
      a.erase(std::unique(a.begin(), a.end()), a.end());
    }
    std::vector<int> perm;
    std::vector<std::vector<int>> spose;
    eliminate(N, adj, ordering == DNLS_ORDER_MIN_DEGREE, perm, spose);
    std::vector<int> iperm(N);
    for (int k = 0; k < N; ++k) iperm[perm[k]] = k;

    // column structure in positions
    std::vector<std::vector<int>> rows(N);
    for (int k = 0; k < N; ++k) {
      for (int v : spose[k]) rows[k].push_back(iperm[v]);
      std::sort(rows[k].begin(), rows[k].end());
    }
    // levels (height above the leaves of the elimination tree; the parent of column k is its
    // first row)
    std::vector<int> lev(N, 0);
    for (int k = 0; k < N; ++k)
      if (!rows[k].empty()) lev[rows[k][0]] = std::max(lev[rows[k][0]], lev[k] + 1);
    int nlev = 0;
    for (int k = 0; k < N; ++k) nlev = std::max(nlev, lev[k] + 1);
    std::vector<std::vector<int>> bylev(nlev);
    for (int k = 0; k < N; ++k) bylev[lev[k]].push_back(k);
    // the top chain: the longest run of one-column levels ending at the root (the columns of
    // the separator eliminated last); its rows' sums over columns outside it are formed in one
    // pass of the forward solve before its levels (at least two such levels, else none)
    int chain_lev = nlev;
    while (chain_lev > 0 && bylev[chain_lev - 1].size() == 1) --chain_lev;
    if (nlev - chain_lev < 2) chain_lev = nlev;
    // algorithmic work on this structure (before any amalgamation): column j with c_j
    // off-diagonal blocks takes part in c_j (c_j + 1) / 2 block updates, c_j of them into
    // diagonal blocks
    int64_t n_upd = 0, n_upd_diag = 0, nnz_alg = 0;
    for (int j = 0; j < N; ++j) {
      const int64_t c = (int64_t)rows[j].size();
      n_upd += c * (c + 1) / 2;
      n_upd_diag += c;
      nnz_alg += c;
    }
    // Supernode amalgamation of the top chain.  Chain column i (level chain_lev + i) has only
    // chain columns above it as rows, and on large pose graphs almost all of them: the chain is
    // the dense trailing block of the factor.  A chain of at least kDenseChainMin columns that
    // holds at least half of its lower-triangle blocks is made fully dense (the missing blocks
    // are explicit zeros: every product that would fill them has a structurally zero factor, so
    // they stay exactly zero) and factored as one dense supernode, right-looking, after the
    // sparse levels.  The parents (first rows) are unchanged, so are the levels.
    int dense_lev = nlev;
    if (dense_chain && nlev - chain_lev >= kDenseChainMin) {
      const int mc = nlev - chain_lev;
      std::vector<int> cc(mc);
      for (int i = 0; i < mc; ++i) cc[i] = bylev[chain_lev + i][0];
      int64_t have = 0;
      bool nested = true;
      for (int i = 0; i < mc; ++i) {
        have += (int64_t)rows[cc[i]].size();
        for (int r : rows[cc[i]]) nested = nested && lev[r] > lev[cc[i]];
        if (i + 1 < mc) nested = nested && cc[i + 1] > cc[i];
      }
      if (nested && 2 * have >= (int64_t)mc * (mc - 1) / 2) {
        for (int i = 0; i < mc; ++i) rows[cc[i]].assign(cc.begin() + i + 1, cc.end());
        dense_lev = chain_lev;
      }
    }
    std::vector<int> colptr(N + 1, 0);
    for (int k = 0; k < N; ++k) colptr[k + 1] = colptr[k] + (int)rows[k].size();
    const int nnzL = colptr[N];
    auto blk = [&](int r, int c) -> int {  // block id of L(r, c), r >= c
      if (r == c) return c;
      auto it = std::lower_bound(rows[c].begin(), rows[c].end(), r);
      if (it == rows[c].end() || *it != r) return -1;
      return N + colptr[c] + (int)(it - rows[c].begin());
    };
    // row structure: for each k, (block L(k, j), j) for j < k
    std::vector<std::vector<std::pair<int, int>>> rowl(N);
    for (int j = 0; j < N; ++j)
      for (int a = 0; a < (int)rows[j].size(); ++a)
        rowl[rows[j][a]].push_back({N + colptr[j] + a, j});
    // gather lists: per target block of column k, the (L(r,j), L(k,j)) pairs, j in rowl[k]; the
    // dense supernode's own products (source column in it) are applied right-looking by the
    // numeric factorization and are not listed
    std::vector<std::vector<std::vector<int>>> gl(N);  // gl[k][t] flat pairs, t=0 diag, 1+a off
    std::vector<std::vector<std::vector<int>>> glv(N);  // level of each pair's source column
    for (int k = 0; k < N; ++k) {
      gl[k].assign(1 + rows[k].size(), {});
      glv[k].assign(1 + rows[k].size(), {});
      for (auto& pr : rowl[k]) {
        const int bkj = pr.first, j = pr.second;
        if (lev[j] >= dense_lev) continue;
        auto it = std::lower_bound(rows[j].begin(), rows[j].end(), k);
        for (; it != rows[j].end(); ++it) {
          const int r = *it;
          const int a_src = N + colptr[j] + (int)(it - rows[j].begin());
          int t;
          if (r == k) {
            t = 0;
          } else {
            auto jt = std::lower_bound(rows[k].begin(), rows[k].end(), r);
            if (jt == rows[k].end() || *jt != r) return DNLS_ERR_ARG;  // cannot happen (closure)
            t = 1 + (int)(jt - rows[k].begin());
          }
          gl[k][t].push_back(a_src);
          gl[k][t].push_back(bkj);
          glv[k][t].push_back(lev[j]);
        }
      }
    }
    // assembly maps
    std::vector<std::vector<int>> inc(N);
    std::map<int, int> pair_of_blk;
    std::vector<std::vector<int>> pairl;
    std::vector<int> pairtgt;
    for (int e = 0; e < E; ++e) {
      int i = edge_i[e0 + e], j = edge_j[e0 + e];
      inc[iperm[i]].push_back(e << 1);
      if (j >= 0) {
        inc[iperm[j]].push_back((e << 1) | 1);
        int pi = iperm[i], pj = iperm[j];
        int R = std::max(pi, pj), C = std::min(pi, pj);
        int id = blk(R, C);
        if (id < 0) return DNLS_ERR_ARG;
        auto f = pair_of_blk.find(id);
        int p;
        if (f == pair_of_blk.end()) {
          p = (int)pairl.size();
          pair_of_blk[id] = p;
          pairl.push_back({});
          pairtgt.push_back(id);
        } else {
          p = f->second;
        }
        pairl[p].push_back((e << 1) | (pi > pj ? 0 : 1));
      }
    }
    const int npair = (int)pairl.size();

    // ---- blob
    ProbMeta& m = G.meta[b];
    m.N = N;
    m.E = E;
    m.npair = npair;
    m.nnzL = nnzL;
    m.nlev = nlev;
    m.n_upd = (int32_t)n_upd;
    m.pose_off = p0;
    m.edge_off = e0;
    m.sym = (int64_t)G.sym.size();
    m.dense_off = dense_off;
    dense_off += (int64_t)N * D * N * D;
    std::vector<int32_t> blob;
    auto mark = [&]() { return (int32_t)blob.size(); };
    m.o_perm = mark();
    blob.insert(blob.end(), perm.begin(), perm.end());
    m.o_iperm = mark();
    blob.insert(blob.end(), iperm.begin(), iperm.end());
    m.o_colptr = mark();
    blob.insert(blob.end(), colptr.begin(), colptr.end());
    m.o_rows = mark();
    for (int k = 0; k < N; ++k) blob.insert(blob.end(), rows[k].begin(), rows[k].end());
    m.o_rowptr = mark();
    {
      int acc = 0;
      for (int k = 0; k < N; ++k) {
        blob.push_back(acc);
        acc += (int)rowl[k].size();
      }
      blob.push_back(acc);
    }
    // within each row, pairs from columns outside the top chain first; rsplit[k] = where the
    // chain columns' pairs begin (the row's end for rows outside the chain)
    std::vector<int32_t> rsplit(N);
    m.o_rowent = mark();
    {
      int acc = 0;
      for (int k = 0; k < N; ++k) {
        int nonchain = 0;
        for (int pass = 0; pass < 2; ++pass)
          for (auto& pr : rowl[k]) {
            if ((lev[pr.second] >= chain_lev) != (pass == 1)) continue;
            blob.push_back(pr.first);
            blob.push_back(pr.second);
            if (pass == 0) ++nonchain;
          }
        rsplit[k] = acc + nonchain;
        acc += (int)rowl[k].size();
      }
    }
    m.o_rsplit = mark();
    blob.insert(blob.end(), rsplit.begin(), rsplit.end());
    m.chain_lev = chain_lev;
    m.dense_lev = dense_lev;
    m.o_lvlptr = mark();
    {
      int acc = 0;
      for (int l = 0; l < nlev; ++l) {
        blob.push_back(acc);
        acc += (int)bylev[l].size();
      }
      blob.push_back(acc);
    }
    m.o_lvlcols = mark();
    for (int l = 0; l < nlev; ++l) blob.insert(blob.end(), bylev[l].begin(), bylev[l].end());
    // targets by level with their gather ranges
    std::vector<int> tgt, gptr, gsrc, tgtptr, pan, panptr, gsplit;
    for (int l = 0; l < nlev; ++l) {
      tgtptr.push_back((int)tgt.size());
      panptr.push_back((int)pan.size() / 2);
      // targets with at least one source pair, longest source list first, so that the
      // threads of a warp run gather loops of similar length (the order of the targets does
      // not change any sum: each target is still summed by one thread group in list order)
      struct LT {
        int count, target, k, t;
      };
      std::vector<LT> lt;
      for (int k : bylev[l])
        for (int t = 0; t <= (int)rows[k].size(); ++t)
          if (!gl[k][t].empty())
            lt.push_back({(int)gl[k][t].size(), t == 0 ? k : N + colptr[k] + t - 1, k, t});
      std::stable_sort(lt.begin(), lt.end(), [](const LT& x, const LT& y) { return x.count > y.count; });
      for (const LT& e : lt) {
        tgt.push_back(e.target);
        gptr.push_back((int)gsrc.size() / 2);
        // "early" pairs first (source column two or more levels below, final once the level
        // below this one has started), then the pairs from the level just below; the order of
        // pairs within each part is kept
        const std::vector<int>& pr = gl[e.k][e.t];
        const std::vector<int>& pl = glv[e.k][e.t];
        // (in the dense supernode every listed pair comes from a sparse column, final before
        // the supernode starts: all of them count as early)
        for (int late = 0; late < 2; ++late) {
          for (int q = 0; q < (int)pl.size(); ++q)
            if ((l < dense_lev && pl[q] >= l - 1) == (late == 1)) {
              gsrc.push_back(pr[2 * q]);
              gsrc.push_back(pr[2 * q + 1]);
            }
          if (late == 0) gsplit.push_back((int)gsrc.size() / 2);
        }
      }
      for (int k : bylev[l]) {
        for (int a = 0; a < (int)rows[k].size(); ++a) {
          pan.push_back(N + colptr[k] + a);
          pan.push_back(k);
        }
      }
    }
    tgtptr.push_back((int)tgt.size());
    panptr.push_back((int)pan.size() / 2);
    gptr.push_back((int)gsrc.size() / 2);
    m.o_tgtptr = mark();
    blob.insert(blob.end(), tgtptr.begin(), tgtptr.end());
    m.o_tgt = mark();
    blob.insert(blob.end(), tgt.begin(), tgt.end());
    m.o_gptr = mark();
    blob.insert(blob.end(), gptr.begin(), gptr.end());
    m.o_gsrc = mark();
    blob.insert(blob.end(), gsrc.begin(), gsrc.end());
    m.o_gsplit = mark();
    blob.insert(blob.end(), gsplit.begin(), gsplit.end());
    m.o_panptr = mark();
    blob.insert(blob.end(), panptr.begin(), panptr.end());
    m.o_pan = mark();
    blob.insert(blob.end(), pan.begin(), pan.end());
    m.o_incptr = mark();
    {
      int acc = 0;
      for (int k = 0; k < N; ++k) {
        blob.push_back(acc);
        acc += (int)inc[k].size();
      }
      blob.push_back(acc);
    }
    m.o_inc = mark();
    for (int k = 0; k < N; ++k) blob.insert(blob.end(), inc[k].begin(), inc[k].end());
    m.o_pairptr = mark();
    {
      int acc = 0;
      for (int p = 0; p < npair; ++p) {
        blob.push_back(acc);
        acc += (int)pairl[p].size();
      }
      blob.push_back(acc);
    }
    m.o_pairs = mark();
    for (int p = 0; p < npair; ++p) blob.insert(blob.end(), pairl[p].begin(), pairl[p].end());
    m.o_pairtgt = mark();
    blob.insert(blob.end(), pairtgt.begin(), pairtgt.end());
    m.o_lsrc = mark();
    {
      std::vector<int32_t> lsrc(nnzL, -1);
      for (int p = 0; p < npair; ++p) lsrc[pairtgt[p] - N] = p;
      blob.insert(blob.end(), lsrc.begin(), lsrc.end());
    }
    // lanes per output element in each level's sums.  Measured on the 128-pose SE(3) graphs:
    // Lanes per output of each level's gather (factor) and sweeps (solves).  A warp issues
    // one FP64 instruction per several dozen cycles, so on levels with few outputs (the top of
    // the elimination tree, where source lists are longest) splitting each output's sum over
    // more lanes shortens the serial chains; on wide levels extra lanes only add instructions.
    // Rule: double the lanes (up to 8) while the level's outputs x lanes still fit in the
    // CTA's threads and each lane keeps at least one term on average.
    const int threads_hint = threads > 0 ? threads : (D == 6 ? 256 : 128);
    auto lanes_for = [&](int64_t outputs, double avg_terms, int min_lanes) {
      int ln = min_lanes;
      while (ln < 8 && outputs * ln * 2 <= threads_hint && avg_terms >= 2.0 * ln) ln *= 2;
      return ln;
    };
    m.o_glanes = mark();
    for (int l = 0; l < nlev; ++l) {
      const int t0 = tgtptr[l], t1 = tgtptr[l + 1];
      const int64_t pairs_l = gptr[t1] - gptr[t0];
      const double avg = t1 > t0 ? (double)pairs_l / (t1 - t0) : 0.0;
      blob.push_back(lanes_for((int64_t)(t1 - t0) * BS, avg, 1));
    }
    {  // glanes[nlev]: the dense supernode's gather of its sparse sources (all its targets)
      const int t0 = tgtptr[dense_lev], t1 = tgtptr[nlev];
      const int64_t pairs_d = gptr[t1] - gptr[t0];
      blob.push_back(t1 > t0 ? lanes_for((int64_t)(t1 - t0) * BS, (double)pairs_d / (t1 - t0), 1) : 1);
    }
    m.o_slanes = mark();
    int64_t pre_terms = 0;  // terms of the top chain's pre-pass
    for (int l = 0; l < nlev; ++l) {
      int64_t fwd = 0, bwd = 0;
      for (int k : bylev[l]) {
        int64_t nonchain = 0;
        for (auto& pr : rowl[k]) nonchain += lev[pr.second] < chain_lev;
        // full row lengths: the same lanes serve solves with and without the chain's pre-pass
        fwd += (int64_t)rowl[k].size();
        if (l >= chain_lev) pre_terms += nonchain;
        bwd += (int64_t)rows[k].size();
      }
      const int nc = (int)bylev[l].size();
      const double avg = nc ? (double)std::max(fwd, bwd) / nc : 0.0;
      blob.push_back(lanes_for((int64_t)nc * D, avg, 1));
    }
    {  // slanes[nlev]: lanes of the top chain's pre-pass
      const int nc = nlev - chain_lev;
      blob.push_back(nc ? lanes_for((int64_t)nc * D, (double)pre_terms / nc, 1) : 1);
    }
    blob.push_back(0);  // keep every section non-empty-addressable
    while (blob.size() % 4) blob.push_back(0);  // 16-byte multiple, for staging copies
    m.blob_len = (int32_t)blob.size();
    G.sym.insert(G.sym.end(), blob.begin(), blob.end());
    // the blob of the next problem must start 16-byte aligned as well
    // (blob lengths are multiples of 4 int32, so every problem's start is)

    // ---- workspace plan (layout independent of the options)
    const int64_t n = (int64_t)N * D;
    const int64_t JW = 2 * BS + D;  // per cost: r, J_i, J_j
    int64_t off = 0;
    auto take = [&](int64_t bytes) {
      int64_t o = off;
      off = align256(off + bytes);
      return (int32_t)o;
    };
    m.w_H = take((int64_t)(N + npair) * BS * 8);
    m.L_bytes = (int32_t)((int64_t)(N + nnzL) * BS * 8);
    m.w_L = take(m.L_bytes);
    m.w_Linv = take((int64_t)N * BS * 8);
    m.w_g = take(n * 8);
    m.w_dx = take(n * 8);
    m.w_tmp = take(n * 8);
    m.w_thc = take((int64_t)N * G.pw * 8);
    m.w_J = take((int64_t)E * JW * 8);
    m.w_bx = take(n * 8);
    m.w_bv = take(n * 8);
    m.w_br = take(n * 8);
    m.w_bhx = take(n * 8);
    m.w_ebuf = take((int64_t)E * 4 * D * 8);
    m.w_state = take(64);
    m.w_W = take((int64_t)E * D * 8);
    m.w_Lf = take((int64_t)(N + nnzL) * BS * 4);
    m.w_Linvf = take((int64_t)N * BS * 4);
    {
      auto a16 = [](int64_t x) { return (x + 15) & ~(int64_t)15; };
      const int64_t arena = a16((int64_t)m.blob_len * 4) + a16(m.L_bytes) + a16((int64_t)N * BS * 8) +
                            2 * a16(n * 8);
      m.arena_bytes = (int32_t)std::min<int64_t>(arena, (int64_t)1 << 30);
    }
    if (off > ((int64_t)1 << 31) - 1) return DNLS_ERR_ARG;
    m.ws = ws;
    ws += off;

    G.max_L_bytes = std::max(G.max_L_bytes, m.L_bytes);
    G.max_arena_bytes = std::max(G.max_arena_bytes, m.arena_bytes);
    G.max_nlev = std::max(G.max_nlev, nlev);
    G.n_blocks_L += N + nnzL;
    G.n_upd += n_upd;
    const double D3 = (double)D * D * D;
    // algorithmic count: an update into a diagonal block needs only its lower triangle
    // (D (D + 1) / 2 outputs; the kernel forms the full block)
    const double ff = 2.0 * (n_upd - n_upd_diag) * D3 + (double)n_upd_diag * D * D * (D + 1) +
                      (double)nnz_alg * D * D * (D + 1) + N * (2.0 * D3 / 3.0);
    G.factor_flops += ff;
    G.prob_flops.push_back(ff);
    G.dense_flops += (double)n * n * n / 3.0;
    cost[b] = ff + 200.0 * E;
  }
  G.ws_bytes = ws;
  G.order.resize(B);
  for (int b = 0; b < B; ++b) G.order[b] = b;
  std::stable_sort(G.order.begin(), G.order.end(),
                   [&](int a, int c) { return cost[a] > cost[c]; });
  return DNLS_OK;
}

}  // namespace dnls
