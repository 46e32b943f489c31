// Host-side planning: circuit -> tensor network, contraction trees, exact
// memoized evaluation counts, slicing, operand layouts and the device program.
#pragma once

#include <algorithm>
#include <array>
#include <complex>
#include <cstdint>
#include <string>
#include <unordered_map>
#include <vector>

#include "xeb.h"

namespace xebp {

using cd = std::complex<double>;

// Thread-local message returned by xeb_last_error().
void set_last_error(const std::string& msg);

// One leaf of the fused circuit network (convention of include/xeb.h).
// Tensor axes: out_q (listed order) then legs; row-major, first axis slowest.
struct Leaf {
    std::vector<int> out_q;
    std::vector<int> legs;
    std::vector<int> qubits;  // qubits of the gate the leaf came from
    std::vector<cd> t;
};

struct Network {
    int n = 0;
    int n_legs = 0;
    std::vector<Leaf> leaves;
    // Multi-batch networks (Sec. "Multi-batch simulator"): the output legs of
    // the qubits in open_mask are left uncontracted.  They are the legs
    // n_legs - n_open .. n_legs - 1, one per open qubit in ascending qubit
    // order (open_legs), each held by a single leaf, so they survive to the
    // root; bond legs keep the ids they have without open qubits.
    uint64_t open_mask = 0;
    int n_open = 0;
    std::vector<int> open_legs;
    bool is_open_leg(int l) const { return l >= n_legs - n_open; }
};

bool build_network(const xeb_circuit* c, Network& net, std::string& err, uint64_t open_mask = 0);

using Tree = std::vector<std::array<int, 2>>;  // post-order (left, right) pairs

// Tensor and index sizes saturate at 2^48 elements (2 PiB of complex64: no
// device holds one), so candidate trees with very wide intermediates cannot
// overflow the planner's integer arithmetic; a plan that reaches the bound
// is refused at bind (XEB_ENOMEM).
constexpr int64_t kSatElems = int64_t(1) << 48;
inline int64_t pow2_sat(size_t b) { return b >= 48 ? kSatElems : int64_t(1) << b; }
inline int64_t mul_sat(int64_t a, int64_t b) {
    if (a <= 0 || b <= 0) return 0;
    return a > kSatElems / b ? kSatElems : std::min(a * b, kSatElems);
}

// Per tree node (uniform ids: leaf j -> j, internal i -> L + i).
struct Node {
    int l = -1, r = -1, parent = -1;
    std::vector<int> legs;  // legs of the node tensor (sliced legs removed)
    int q = 0;              // legs summed at this node (internal)
    uint64_t qmask = 0;     // output qubits the subtree depends on
    int a = 0, b = 0;       // range in pi
    int64_t kv = 1;         // exact number of distinct values of its bits
};

struct Analysis {
    int L = 0;
    std::vector<Node> nodes;
    std::vector<int> pi;
};

// Distinct-count oracle over the plan's bitstrings, cached by qubit mask.
struct DistinctCounter {
    const uint64_t* bs = nullptr;
    size_t k = 0;
    std::unordered_map<uint64_t, int64_t> cache;
    std::vector<uint64_t> scratch;
    int64_t count(uint64_t mask);
};

bool check_tree(const Tree& t, int n_leaves, std::string& err);
// Commutativity (App. A): put the child with more free (unshared, unsliced)
// legs on the left of every node, so each contraction has M >= N (the left
// child is the A operand).  Costs are unchanged; only the in-order bit order
// and the operand roles change.
void orient_tree(const Network& net, Tree& t, const std::vector<int>& sliced);
bool analyze(const Network& net, const Tree& tree, const std::vector<int>& sliced,
             Analysis& an, std::string& err);
void fill_counts(Analysis& an, DistinctCounter& dc);

// ---- device program ----------------------------------------------------------
enum OpKind { OP_PERM = 1, OP_GEMM = 2 };

struct Op {
    int kind = 0;
    int node = -1;          // uniform id of the node produced (GEMM) / permuted (PERM)
    // PERM: dst[key][x'] = src[key][x] where dst bit j comes from src bit perm[j]
    int src_buf = -1, dst_buf = -1;
    int r = 0;
    int64_t keys = 0;
    std::vector<int> perm;
    // GEMM: for u < kv: C_u = A_{uL(u)} (M x K) * B_{uR(u)} (K x N)
    int a_buf = -1, b_buf = -1, c_buf = -1;
    int a_node = -1, b_node = -1;
    int64_t M = 1, N = 1, K = 1, kv = 1;
    // operand addressing: bit i of the row / summed / column index sits at
    // address bit pos[i] of the operand tensor (legs have dimension 2)
    std::vector<int> a_pos_m, a_pos_k, b_pos_k, b_pos_n;
    int a_rank = 0, b_rank = 0;
    // output addressing: bit i of m / n sits at address bit c_pos_m[i] /
    // c_pos_n[i] of the result (row-major [M][N] when natural)
    std::vector<int> c_pos_m, c_pos_n;
    std::vector<int> c_hint;  // legs of this result that its parent sums (low bits)
};

struct Buffer {
    int64_t elems = 0;   // complex elements
    int64_t off = -1;    // element offset in the arena
    int first = -1, last = -1;
};

struct Program {
    std::vector<Op> ops;
    std::vector<Buffer> bufs;
    std::vector<int> node_buf;                 // final buffer of each node's tensor
    std::vector<std::vector<int>> layout;      // stored leg order per node (slowest first)
    int64_t arena_elems = 0;
    double permute_elems = 0;
};

// gather = true: contractions read their operands in place through per-leg
// address positions (no permutation passes); false: permute operands into
// [free][summed] blocks first.
// consumer_layout = true: a result of >= 2^20 elements is laid out with the
// legs its parent sums as the lowest address bits, so the parent reads whole
// contiguous rows.
void build_program(const Analysis& an, Program& prog, bool gather, bool consumer_layout = false);
void plan_memory(Program& prog);  // emulation-mode allocator: exact arena peak

struct Costs {
    double C = 0, RW = 0, single = 0, perm = 0;
};
Costs tree_costs(const Analysis& an, const Program& prog, uint64_t k);

// Contractions the tcgen05 split-precision kernel takes: one key, 128-row
// tiles, 16 <= K, N <= 64 complex.
inline bool tc_eligible(const Op& op) {
    return op.kind == OP_GEMM && op.kv == 1 && op.M >= 128 && op.M % 128 == 0 && op.K >= 16 && op.K <= 64 &&
           op.N >= 16 && op.N <= 64;
}

// Estimated device time of one slice (seconds) from a simple efficiency
// profile of GB300: per contraction max(flop time, HBM time) + launch cost.
// The objective uses log2 of it in place of log2(C + alpha RW) (App. A, last
// paragraph of "Slicing": a measured efficiency profile replaces the flop and
// read/write counts).
double estimate_time(const Analysis& an, const Program& prog, int precision, size_t elem);

// The same efficiency profile for one contraction of `cmac` complex MACs that
// moves `bytes` through HBM, on the tensor cores or the SIMT cores.
double contraction_time(double cmac, double bytes, bool tensor_core, int precision);

// Expected number of distinct values of b uniform random bits among k draws,
// 2^b (1 - (1 - 2^-b)^k) (never above the App. C bound min(2^b, k)).
double expected_distinct(int b, uint64_t k);

// ---- planners ----------------------------------------------------------------
Tree greedy_tree(const Network& net, DistinctCounter& dc, const std::vector<int>& sliced,
                 uint64_t seed, double noise);
// variant 0: blocks grow while consecutive gates fit in block_qubits qubits;
// variant 1: frontier blocks -- a window of <= block_qubits qubits absorbs
// every gate whose predecessors are done, then widens by the earliest ready
// gate that still fits.
bool sweep_tree(const Network& net, int block_qubits, int group_leaves, Tree& out, int variant = 0);

// Local search over contraction trees and slice sets (App. A): simulated
// annealing with the four rewrites (a*b)*c -> (c*b)*a, (a*b)*c -> (a*c)*b,
// a*(b*c) -> c*(b*a), a*(b*c) -> b*(a*c), whose gain is computed locally
// (App. C: only the rewritten node and its parent change), and every
// `slice_every` proposals a slicing move: add the leg with the best memory
// reduction while over budget, else drop a random sliced leg.  The objective
// is f = beta max(log2(M / M_max), 0) + |S| + log2 T with T the efficiency-
// profile time of one slice and M = 2 (sum_v m_v^p)^(1/p), m_v = k_v 2^{r_v}
// elements of node v (App. C's p-norm estimate of the largest live tensors).
// During the search k_v is expected_distinct(|B_v|, k).
struct AnnealOpts {
    int64_t steps = 0;
    int64_t slice_every = 0;   // 0: the slice set stays as given
    double t0 = 0.5, t1 = 0.005;
    double beta = 10.0;
    double budget_elems = 1;   // M_max in complex elements
    double p = 8.0;
    int precision = XEB_PREC_FP32;
    size_t elem = 8;
    uint64_t seed = 1;
    int max_sliced = 30;
};
struct AnnealStats {
    double f_start = 0, f_best = 0;
    int64_t accepted = 0;
};
// Refines (tree, sliced) in place to the best state visited.
void anneal_tree(const Network& net, uint64_t k, Tree& tree, std::vector<int>& sliced, const AnnealOpts& ao,
                 AnnealStats* stats = nullptr);
// Independent restarts, one per start tree (seed derived from ao.seed and the
// restart index, so the result does not depend on the number of host threads
// that run them); each tree and slice set is refined in place.
void anneal_many(const Network& net, uint64_t k, std::vector<Tree>& trees, std::vector<std::vector<int>>& sliced,
                 const AnnealOpts& ao, std::vector<AnnealStats>& stats);

}  // namespace xebp
