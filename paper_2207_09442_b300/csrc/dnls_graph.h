// Host/device shared layout of a pose-graph batch handle: per-problem metadata, the symbolic
// block-Cholesky structure and the workspace plan.  Built once per structure on the host
// (dnls_symbolic.cpp) and uploaded; the kernels (dnls_graph.cu) only read it.
#pragma once

#include <cstdint>
#include <vector>

namespace dnls {

// Per-problem metadata.  All o_* fields are int32 offsets into the symbolic blob relative to
// `sym`; all w_* fields are byte offsets into the workspace relative to `ws`.
//
// Block numbering of the factor L (positions = block columns after the fill-reducing
// permutation): diagonal block of position k has id k; the a-th off-diagonal block of column k
// (row position rows[colptr[k] + a]) has id N + colptr[k] + a.  Every block is a dense DOFxDOF
// row-major FP64 matrix.  H keeps the undamped normal matrix: diagonal blocks 0..N-1 and one
// block per distinct connected pose pair (id N + pair).
struct ProbMeta {
  int32_t N, E, npair, nnzL;
  int32_t nlev, n_upd;
  int64_t pose_off, edge_off;  // offsets of this problem in the caller's pose / cost arrays
  int64_t sym;                 // int32 index of this problem's symbolic data in the blob
  int64_t ws;                  // byte offset of this problem's workspace region
  int64_t dense_off;           // offset of this problem's dense n x n block (linearize output)
  int32_t o_perm, o_iperm;     // [N] position -> pose, pose -> position
  int32_t o_colptr, o_rows;    // [N+1], [nnzL]: column structure (row positions, ascending)
  int32_t o_rowptr, o_rowent;  // [N+1], [2 nnzL]: row structure, pairs (block id, column j)
  int32_t o_lvlptr, o_lvlcols; // [nlev+1], [N]: columns grouped by elimination-tree level
  int32_t o_tgtptr, o_tgt;     // [nlev+1], [N + nnzL]: factor target blocks grouped by level
  int32_t o_gptr, o_gsrc;      // [N + nnzL + 1] (parallel to tgt), [2 x pairs]: source pairs
  int32_t o_panptr, o_pan;     // [nlev+1], [2 nnzL]: (off-diagonal block, column) by level
  int32_t o_incptr, o_inc;     // [N+1] by position, [incidences]: cost << 1 | slot
  int32_t o_pairptr, o_pairs;  // [npair+1], [n_between]: cost << 1 | orientation
  int32_t o_pairtgt, o_lsrc;   // [npair]: L block id of each pair; [nnzL]: pair of each L block or -1
  int32_t o_glanes, o_slanes;  // [nlev + 1], [nlev + 1]: lanes per output in the level's gathers /
                               // solve sweeps (1, 2, 4 or 8); glanes[nlev]: the dense supernode's
                               // gather of its sparse sources
  int32_t o_gsplit, o_rsplit;  // [N + nnzL] (parallel to tgt): end of the target's "early" source
                               // pairs (columns two or more levels below), which come first;
                               // [N]: start of row k's pairs from top-chain columns (rowent)
  int32_t chain_lev;           // first level of the top chain (nlev: none); slanes[nlev] holds
                               // the lanes of its pre-pass
  int32_t dense_lev;           // first level of the dense supernode (nlev: none): the top chain
                               // amalgamated into one dense block (explicit zero blocks added),
                               // factored right-looking after the sparse levels; its targets'
                               // source lists hold only the pairs from sparse columns
  int32_t w_H, w_L, w_Linv;    // workspace byte offsets
  int32_t w_g, w_dx, w_tmp, w_thc, w_J;
  int32_t w_bx, w_bv, w_br, w_bhx, w_ebuf, w_state, w_W;
  int32_t w_Lf, w_Linvf;       // FP32 copies of L and the inverted diagonal blocks (mixed-path
                               // forward solves)
  int32_t L_bytes;             // bytes of this problem's factor storage
  int32_t blob_len;            // int32 count of this problem's symbolic data
  int32_t arena_bytes;         // shared memory to stage blob + L + L^-1 + two solve vectors
};

// Mutable per-problem state kept in the workspace between forward and backward.
struct ProbState {
  double lambda_fact;  // damping of the cached factorization
  double S;            // objective at the returned poses
  int32_t factor_ok;   // cached factorization valid
  int32_t fact_flag;   // failed-pivot flag of a cluster factorization (the LM iteration's number)
  int32_t pad[2];
};

struct GraphHost {
  int kind, dof, pw, B;
  int64_t P_total, E_total;
  std::vector<ProbMeta> meta;
  std::vector<int32_t> sym;
  std::vector<int32_t> order;  // problems, most expensive first
  std::vector<int32_t> ei, ej;
  int64_t ws_bytes;            // total workspace bytes (header + problem regions)
  int32_t max_L_bytes, max_nlev, max_arena_bytes;
  int64_t n_blocks_L, n_upd;
  double factor_flops, dense_flops;
  std::vector<double> prob_flops;  // FP64 flops of one numeric factorization, per problem
};

// Workspace header (first bytes of the workspace): the persistent launches' work counters.
constexpr int64_t kWsHeader = 256;

// Returns 0 on success, or a DNLS_ERR_* code; fills `out`.
// `threads` = the threads that will run one problem's factorization (0: one CTA's default),
// used to choose the lanes per output of each level's sums.
// `dense_chain`: amalgamate a long, mostly dense top chain into one dense supernode (pose
// graphs); the bundle-adjustment reduced system (factored by a cluster of CTAs) keeps the level
// schedule throughout.
int build_graph_host(int kind, int B, const int64_t* pose_offsets, const int64_t* edge_offsets,
                     const int32_t* edge_i, const int32_t* edge_j, int ordering, GraphHost* out,
                     int threads = 0, bool dense_chain = true);

// Smallest top chain (block columns) amalgamated into a dense supernode.
constexpr int kDenseChainMin = 32;

}  // namespace dnls
