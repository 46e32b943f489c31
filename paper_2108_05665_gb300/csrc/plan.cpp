// Host-side planning.  See plan.h.
//
// * build_network: circuit -> tensor network N_C with n open legs, gate fusion
//   applied (Sec. "Multi-batch simulator"), in the leaf/leg convention of
//   include/xeb.h.
// * analyze / fill_counts: per tree node, its tensor legs, the legs it sums
//   (q), the output bits it depends on (a contiguous range of the in-order bit
//   order pi) and its exact evaluation count k_v = number of distinct values
//   of those bits among the bitstrings (App. C, "Complexity estimation": a
//   subexpression is evaluated once per distinct value of its variables).
// * build_program: operand layouts for every pairwise contraction T*S
//   (Eq. elem-cont) as a GEMM per key, with leg permutations where a child's
//   stored order does not split into [free][summed] blocks.
// * plan_memory: the "emulation mode" of App. C -- run the schedule with a
//   virtual first-fit allocator to get the exact peak memory.
// * tree_costs: C = sum_v k_v 2^(q_v + r_v) and RW = sum_v k_v (m(L) + m(R) +
//   m(v)) (App. A/C), the single-amplitude cost k * sum_v 2^(q_v + r_v) and the
//   elements our layout permutations move.
// * greedy_tree / sweep_tree: candidate trees for the objective of App. A.
#include "plan.h"

#include <algorithm>
#include <cmath>
#include <functional>
#include <map>
#include <random>
#include <set>

namespace xebp {

// ---- tensor helpers (axis a of a rank-r tensor is bit r-1-a of the index) ----

static void apply_on_axis(std::vector<cd>& t, int rank, int ax, const cd m[4]) {
    const int64_t size = int64_t(1) << rank;
    const int64_t s = int64_t(1) << (rank - 1 - ax);
    for (int64_t x = 0; x < size; ++x) {
        if (x & s) continue;
        const cd a0 = t[x], a1 = t[x | s];
        t[x] = m[0] * a0 + m[1] * a1;
        t[x | s] = m[2] * a0 + m[3] * a1;
    }
}

static std::vector<cd> contract_axis(const std::vector<cd>& t, int rank, int ax, const cd v[2]) {
    const int bit = rank - 1 - ax;
    const int64_t s = int64_t(1) << bit;
    std::vector<cd> r(size_t(1) << (rank - 1));
    for (int64_t y = 0; y < int64_t(r.size()); ++y) {
        const int64_t x = ((y >> bit) << (bit + 1)) | (y & (s - 1));
        r[y] = t[x] * v[0] + t[x | s] * v[1];
    }
    return r;
}

static std::vector<cd> transpose_axes(const std::vector<cd>& t, int rank, const std::vector<int>& order) {
    // new axis i = old axis order[i]
    std::vector<cd> r(t.size());
    for (int64_t y = 0; y < int64_t(t.size()); ++y) {
        int64_t x = 0;
        for (int i = 0; i < rank; ++i) {
            const int64_t bit = (y >> (rank - 1 - i)) & 1;
            x |= bit << (rank - 1 - order[i]);
        }
        r[y] = t[x];
    }
    return r;
}

// ---- circuit -> network -------------------------------------------------------

namespace {
enum LabKind { LAB_OUT = 0, LAB_IN = 1, LAB_LEG = 2, LAB_BIT = 3 };
struct RawLeaf {
    std::vector<cd> t;
    std::vector<std::pair<int, int>> lab;
    std::vector<int> qubits;
};
int find_label(const RawLeaf& r, int kind, int id) {
    for (size_t i = 0; i < r.lab.size(); ++i)
        if (r.lab[i].first == kind && r.lab[i].second == id) return int(i);
    return -1;
}
}  // namespace

bool build_network(const xeb_circuit* c, Network& net, std::string& err, uint64_t open_mask) {
    if (!c) { err = "circuit is NULL"; return false; }
    const int n = c->n_qubits;
    if (n < 1 || n > 64) { err = "n_qubits must be in [1, 64]"; return false; }
    if (n < 64 && (open_mask >> n) != 0) { err = "open qubit above n"; return false; }
    if (c->n_gates < 0 || (c->n_gates > 0 && (!c->kinds || !c->q0 || !c->mats))) {
        err = "circuit arrays missing";
        return false;
    }
    std::vector<std::array<cd, 2>> init(n, {cd(1, 0), cd(0, 0)});
    std::vector<int> last(n, -1);
    std::vector<RawLeaf> raw;
    int next_leg = 0;
    for (int g = 0; g < c->n_gates; ++g) {
        const double* m = c->mats + size_t(g) * 32;
        auto M = [&](int i, int j) { return cd(m[(i * 4 + j) * 2], m[(i * 4 + j) * 2 + 1]); };
        const int kind = c->kinds[g];
        const int a = c->q0[g];
        if (a < 0 || a >= n) { err = "gate " + std::to_string(g) + ": qubit out of range"; return false; }
        if (kind == 1) {
            const cd m2[4] = {M(0, 0), M(0, 1), M(1, 0), M(1, 1)};
            if (last[a] < 0) {
                const cd v0 = m2[0] * init[a][0] + m2[1] * init[a][1];
                const cd v1 = m2[2] * init[a][0] + m2[3] * init[a][1];
                init[a] = {v0, v1};
            } else {
                RawLeaf& p = raw[last[a]];
                apply_on_axis(p.t, int(p.lab.size()), find_label(p, LAB_OUT, a), m2);
            }
            continue;
        }
        if (kind != 2) { err = "gate " + std::to_string(g) + ": kind must be 1 or 2"; return false; }
        if (!c->q1) { err = "q1 missing"; return false; }
        const int b = c->q1[g];
        if (b < 0 || b >= n || b == a) { err = "gate " + std::to_string(g) + ": bad second qubit"; return false; }
        RawLeaf lf;
        lf.t.resize(16);
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j) lf.t[i * 4 + j] = M(i, j);  // [oa][ob][ia][ib]
        lf.lab = {{LAB_OUT, a}, {LAB_OUT, b}, {LAB_IN, a}, {LAB_IN, b}};
        lf.qubits = {a, b};
        for (int s : {a, b}) {
            const int ax = find_label(lf, LAB_IN, s);
            if (last[s] < 0) {
                const cd v[2] = {init[s][0], init[s][1]};
                lf.t = contract_axis(lf.t, int(lf.lab.size()), ax, v);
                lf.lab.erase(lf.lab.begin() + ax);
            } else {
                RawLeaf& p = raw[last[s]];
                p.lab[find_label(p, LAB_OUT, s)] = {LAB_LEG, next_leg};
                lf.lab[ax] = {LAB_LEG, next_leg};
                ++next_leg;
            }
        }
        raw.push_back(std::move(lf));
        last[a] = last[b] = int(raw.size()) - 1;
    }
    // output side of every qubit: projected on the bitstring's bit, or (open
    // qubits) a leg of its own, numbered after all bond legs
    const int n_bond = next_leg;
    net.open_legs.clear();
    for (int q = 0; q < n; ++q) {
        const bool open = (open_mask >> q) & 1;
        const std::pair<int, int> lab = open ? std::pair<int, int>{LAB_LEG, next_leg} : std::pair<int, int>{LAB_BIT, q};
        if (open) net.open_legs.push_back(next_leg++);
        if (last[q] < 0) {
            RawLeaf lf;
            lf.t = {init[q][0], init[q][1]};
            lf.lab = {lab};
            lf.qubits = {q};
            raw.push_back(std::move(lf));
        } else {
            RawLeaf& p = raw[last[q]];
            p.lab[find_label(p, LAB_OUT, q)] = lab;
        }
    }
    net.n = n;
    net.n_legs = next_leg;
    net.open_mask = open_mask;
    net.n_open = next_leg - n_bond;
    net.leaves.clear();
    for (RawLeaf& r : raw) {
        Leaf lf;
        std::vector<int> order;
        for (size_t i = 0; i < r.lab.size(); ++i)
            if (r.lab[i].first == LAB_BIT) { order.push_back(int(i)); lf.out_q.push_back(r.lab[i].second); }
        for (size_t i = 0; i < r.lab.size(); ++i)
            if (r.lab[i].first == LAB_LEG) { order.push_back(int(i)); lf.legs.push_back(r.lab[i].second); }
        if (order.size() != r.lab.size()) { err = "internal: unresolved label"; return false; }
        lf.t = transpose_axes(r.t, int(order.size()), order);
        lf.qubits = r.qubits;
        net.leaves.push_back(std::move(lf));
    }
    return true;
}

// ---- tree analysis --------------------------------------------------------------

bool check_tree(const Tree& t, int L, std::string& err) {
    if (L < 2) { err = "network needs at least two leaves"; return false; }
    if (int(t.size()) != L - 1) { err = "tree must have n_leaves - 1 nodes"; return false; }
    std::vector<int> seen_leaf(L, 0), used(t.size(), 0);
    for (size_t i = 0; i < t.size(); ++i) {
        for (int c : t[i]) {
            if (c < 0) {
                const int j = -1 - c;
                if (j >= L) { err = "tree references leaf out of range"; return false; }
                if (seen_leaf[j]++) { err = "leaf used twice in tree"; return false; }
            } else {
                if (c >= int(i)) { err = "tree children must precede their parent"; return false; }
                if (used[c]++) { err = "tree node used twice"; return false; }
            }
        }
    }
    for (size_t i = 0; i + 1 < t.size(); ++i)
        if (!used[i]) { err = "tree node without parent"; return false; }
    return true;
}

bool analyze(const Network& net, const Tree& tree, const std::vector<int>& sliced, Analysis& an,
             std::string& err) {
    const int L = int(net.leaves.size());
    if (!check_tree(tree, L, err)) return false;
    std::vector<char> is_sliced(net.n_legs, 0);
    for (int l : sliced) {
        if (l < 0 || l >= net.n_legs) { err = "sliced leg out of range"; return false; }
        if (is_sliced[l]) { err = "sliced leg listed twice"; return false; }
        if (net.is_open_leg(l)) { err = "an open output leg cannot be sliced"; return false; }
        is_sliced[l] = 1;
    }
    an.L = L;
    an.nodes.assign(L + tree.size(), Node());
    for (int j = 0; j < L; ++j) {
        Node& nd = an.nodes[j];
        for (int l : net.leaves[j].legs)
            if (!is_sliced[l]) nd.legs.push_back(l);
        for (int q : net.leaves[j].out_q) nd.qmask |= uint64_t(1) << q;
    }
    std::vector<char> mark(net.n_legs, 0);
    for (size_t i = 0; i < tree.size(); ++i) {
        const int v = L + int(i);
        Node& nd = an.nodes[v];
        nd.l = tree[i][0] < 0 ? -1 - tree[i][0] : L + tree[i][0];
        nd.r = tree[i][1] < 0 ? -1 - tree[i][1] : L + tree[i][1];
        Node& A = an.nodes[nd.l];
        Node& B = an.nodes[nd.r];
        A.parent = B.parent = v;
        for (int l : B.legs) mark[l] = 1;
        nd.q = 0;
        for (int l : A.legs) {
            if (mark[l]) ++nd.q;
            else nd.legs.push_back(l);
        }
        for (int l : B.legs) mark[l] = 0;
        for (int l : A.legs) mark[l] = 1;
        for (int l : B.legs)
            if (!mark[l]) nd.legs.push_back(l);
        for (int l : A.legs) mark[l] = 0;
        nd.qmask = A.qmask | B.qmask;
        if (nd.legs.size() > 48) { err = "tensor with more than 48 legs"; return false; }
    }
    // pi and ranges by an in-order walk
    an.pi.clear();
    std::function<void(int)> walk = [&](int v) {
        Node& nd = an.nodes[v];
        if (v < L) {
            nd.a = int(an.pi.size());
            for (int q : net.leaves[v].out_q) an.pi.push_back(q);
            nd.b = int(an.pi.size());
            return;
        }
        walk(nd.l);
        walk(nd.r);
        nd.a = an.nodes[nd.l].a;
        nd.b = an.nodes[nd.r].b;
    };
    walk(L + int(tree.size()) - 1);
    if (int(an.pi.size()) != net.n - net.n_open) { err = "internal: pi is not a permutation"; return false; }
    return true;
}

void orient_tree(const Network& net, Tree& t, const std::vector<int>& sliced) {
    const int L = int(net.leaves.size());
    std::set<int> sl(sliced.begin(), sliced.end());
    std::vector<std::vector<int>> legs(t.size());  // internal node legs, sorted
    auto legs_of = [&](int ref) -> std::vector<int> {
        if (ref >= 0) return legs[ref];
        std::vector<int> v;
        for (int l : net.leaves[-1 - ref].legs)
            if (!sl.count(l)) v.push_back(l);
        std::sort(v.begin(), v.end());
        return v;
    };
    (void)L;
    for (size_t i = 0; i < t.size(); ++i) {
        const std::vector<int> a = legs_of(t[i][0]), b = legs_of(t[i][1]);
        std::vector<int> shared, x;
        std::set_intersection(a.begin(), a.end(), b.begin(), b.end(), std::back_inserter(shared));
        std::set_symmetric_difference(a.begin(), a.end(), b.begin(), b.end(), std::back_inserter(x));
        legs[i] = x;
        if (b.size() > a.size()) std::swap(t[i][0], t[i][1]);
    }
}

int64_t DistinctCounter::count(uint64_t mask) {
    if (mask == 0 || k == 0) return 1;
    auto it = cache.find(mask);
    if (it != cache.end()) return it->second;
    scratch.resize(k);
    for (size_t i = 0; i < k; ++i) scratch[i] = bs[i] & mask;
    std::sort(scratch.begin(), scratch.end());
    const int64_t c = std::unique(scratch.begin(), scratch.end()) - scratch.begin();
    cache.emplace(mask, c);
    return c;
}

void fill_counts(Analysis& an, DistinctCounter& dc) {
    for (Node& nd : an.nodes) nd.kv = dc.count(nd.qmask);
}

// ---- program: layouts, permutations, GEMMs ----------------------------------------

namespace {
// Split `lay` into (F, sigma): returns 0 for [F][S] (S lowest bits), 1 for
// [S][F], -1 if S is not a contiguous block at either end.
int split_kind(const std::vector<int>& lay, const std::vector<char>& inS, std::vector<int>& sigma,
               std::vector<int>& F) {
    sigma.clear();
    F.clear();
    for (int l : lay) (inS[l] ? sigma : F).push_back(l);
    if (sigma.empty() || F.empty()) return 0;
    const size_t ns = sigma.size();
    bool tail = true, head = true;
    for (size_t i = 0; i < ns; ++i) {
        if (!inS[lay[lay.size() - 1 - i]]) tail = false;
        if (!inS[lay[i]]) head = false;
    }
    if (tail) return 0;
    if (head) return 1;
    return -1;
}

std::vector<int> concat(const std::vector<int>& a, const std::vector<int>& b) {
    std::vector<int> r(a);
    r.insert(r.end(), b.begin(), b.end());
    return r;
}
}  // namespace

void build_program(const Analysis& an, Program& prog, bool gather, bool consumer_layout) {
    const int N = int(an.nodes.size());
    const int L = an.L;
    int n_legs = 0;
    for (const Node& nd : an.nodes)
        for (int l : nd.legs) n_legs = std::max(n_legs, l + 1);
    prog = Program();
    prog.node_buf.assign(N, -1);
    prog.layout.assign(N, {});
    auto new_buf = [&](int64_t elems, int first) {
        Buffer b;
        b.elems = elems;
        b.first = first;
        b.last = first;
        prog.bufs.push_back(b);
        return int(prog.bufs.size()) - 1;
    };
    auto elems_of = [&](int v) { return mul_sat(an.nodes[v].kv, pow2_sat(an.nodes[v].legs.size())); };
    // leaves are materialised in their canonical leg order
    for (int j = 0; j < L; ++j) {
        prog.layout[j] = an.nodes[j].legs;
        prog.node_buf[j] = new_buf(elems_of(j), 0);
    }
    std::vector<char> inS(std::max(n_legs, 1), 0);
    std::vector<int> s1, f1, s2, f2;
    // legs each node's parent sums (the node's share of its parent's K)
    std::vector<std::vector<int>> summed_by_parent(N);
    for (int v = L; v < N; ++v) {
        const Node& nd = an.nodes[v];
        std::vector<int> S;
        for (int l : an.nodes[nd.l].legs)
            if (std::find(an.nodes[nd.r].legs.begin(), an.nodes[nd.r].legs.end(), l) != an.nodes[nd.r].legs.end())
                S.push_back(l);
        summed_by_parent[nd.l] = S;
        summed_by_parent[nd.r] = S;
    }
    // address bit of `leg` in layout `lay` (slowest first)
    auto pos_of = [](const std::vector<int>& lay, int leg) {
        const int i = int(std::find(lay.begin(), lay.end(), leg) - lay.begin());
        return int(lay.size()) - 1 - i;
    };
    for (int v = L; v < N; ++v) {
        const Node& nd = an.nodes[v];
        const int c1 = nd.l, c2 = nd.r;
        for (int l : an.nodes[c2].legs) inS[l] = 1;
        std::vector<int> S;
        for (int l : an.nodes[c1].legs)
            if (inS[l]) S.push_back(l);
        for (int l : an.nodes[c2].legs) inS[l] = 0;
        for (int l : S) inS[l] = 1;
        auto permute_to = [&](int c, const std::vector<int>& lay) {
            Op op;
            op.kind = OP_PERM;
            op.node = c;
            op.src_buf = prog.node_buf[c];
            op.r = int(lay.size());
            op.keys = an.nodes[c].kv;
            const std::vector<int>& old = prog.layout[c];
            op.perm.assign(op.r, 0);
            for (int j = 0; j < op.r; ++j) op.perm[j] = pos_of(old, lay[op.r - 1 - j]);
            const int idx = int(prog.ops.size()) + 1;
            op.dst_buf = new_buf(elems_of(c), idx);
            prog.bufs[op.src_buf].last = std::max(prog.bufs[op.src_buf].last, idx);
            prog.node_buf[c] = op.dst_buf;
            prog.layout[c] = lay;
            prog.permute_elems += 2.0 * double(elems_of(c));
            prog.ops.push_back(op);
        };
        if (!gather) {
            const int k1 = split_kind(prog.layout[c1], inS, s1, f1);
            const int k2 = split_kind(prog.layout[c2], inS, s2, f2);
            if (k1 >= 0 && k2 >= 0) {
                if (s1 != s2) {
                    if (elems_of(c1) <= elems_of(c2))
                        permute_to(c1, k1 == 0 ? concat(f1, s2) : concat(s2, f1));
                    else
                        permute_to(c2, k2 == 1 ? concat(s1, f2) : concat(f2, s1));
                }
            } else if (k1 >= 0) {
                permute_to(c2, concat(s1, f2));
            } else if (k2 >= 0) {
                permute_to(c1, concat(f1, s2));
            } else {
                const std::vector<int>& sig = elems_of(c1) >= elems_of(c2) ? s1 : s2;
                permute_to(c1, concat(f1, sig));
                permute_to(c2, concat(sig, f2));
            }
        }
        const std::vector<int>& la = prog.layout[c1];
        const std::vector<int>& lb = prog.layout[c2];
        Op op;
        op.kind = OP_GEMM;
        op.node = v;
        op.a_node = c1;
        op.b_node = c2;
        op.a_buf = prog.node_buf[c1];
        op.b_buf = prog.node_buf[c2];
        op.a_rank = int(la.size());
        op.b_rank = int(lb.size());
        // rows: A's free legs in ascending address order; summed index: the
        // shared legs in ascending A address order; columns: B's free legs in
        // ascending B address order
        std::vector<int> fa, fb, sg;
        for (int b = 0; b < op.a_rank; ++b) {
            const int leg = la[op.a_rank - 1 - b];
            if (inS[leg]) { sg.push_back(leg); op.a_pos_k.push_back(b); }
            else { fa.push_back(leg); op.a_pos_m.push_back(b); }
        }
        for (int leg : sg) op.b_pos_k.push_back(pos_of(lb, leg));
        for (int b = 0; b < op.b_rank; ++b) {
            const int leg = lb[op.b_rank - 1 - b];
            if (!inS[leg]) { fb.push_back(leg); op.b_pos_n.push_back(b); }
        }
        op.M = pow2_sat(fa.size());
        op.N = pow2_sat(fb.size());
        op.K = pow2_sat(sg.size());
        op.kv = nd.kv;
        const int idx = int(prog.ops.size()) + 1;
        op.c_buf = new_buf(elems_of(v), idx);
        prog.bufs[op.a_buf].last = std::max(prog.bufs[op.a_buf].last, idx);
        prog.bufs[op.b_buf].last = std::max(prog.bufs[op.b_buf].last, idx);
        prog.node_buf[v] = op.c_buf;
        // C = [rows][cols] row-major: slowest-first layout is the reverse of
        // the ascending address order
        std::vector<int> lay;
        for (size_t t = fa.size(); t-- > 0;) lay.push_back(fa[t]);
        std::vector<int> lc;
        for (size_t t = fb.size(); t-- > 0;) lc.push_back(fb[t]);
        std::vector<int> out = concat(lay, lc);
        if (gather && consumer_layout && v != N - 1 && elems_of(v) >= (int64_t(1) << 20) &&
            !summed_by_parent[v].empty() && summed_by_parent[v].size() <= 6 && tc_eligible(op)) {
            // stable partition: the legs the parent sums move to the lowest bits
            const std::vector<int>& sp = summed_by_parent[v];
            auto in_sp = [&](int leg) { return std::find(sp.begin(), sp.end(), leg) != sp.end(); };
            std::vector<int> hi, lo;
            for (int leg : out) (in_sp(leg) ? lo : hi).push_back(leg);
            out = concat(hi, lo);
            op.c_hint = sp;
        }
        prog.layout[v] = out;
        for (int leg : fa) op.c_pos_m.push_back(pos_of(out, leg));
        for (int leg : fb) op.c_pos_n.push_back(pos_of(out, leg));
        prog.ops.push_back(op);
        for (int l : S) inS[l] = 0;
    }
    // the root tensor is read after the last op (cross-slice accumulation)
    prog.bufs[prog.node_buf[N - 1]].last = int(prog.ops.size()) + 1;
}

void plan_memory(Program& prog) {
    const int64_t align = 64;  // elements
    const int T = int(prog.ops.size()) + 2;
    std::vector<std::vector<int>> born(T), dies(T);
    for (size_t i = 0; i < prog.bufs.size(); ++i) {
        born[prog.bufs[i].first].push_back(int(i));
        dies[std::min(prog.bufs[i].last, T - 1)].push_back(int(i));
    }
    std::map<int64_t, int64_t> live;  // offset -> length
    int64_t peak = 0;
    for (int t = 0; t < T; ++t) {
        for (int bi : born[t]) {
            const int64_t len = (std::min(prog.bufs[bi].elems, kSatElems) + align - 1) / align * align;
            int64_t pos = 0;
            for (auto& kv : live) {
                if (kv.first - pos >= len) break;
                pos = std::max(pos, kv.first + kv.second);
            }
            live.emplace(pos, len);
            prog.bufs[bi].off = pos;
            peak = std::max(peak, pos + len);
        }
        for (int bi : dies[t]) live.erase(prog.bufs[bi].off);
    }
    prog.arena_elems = std::min(peak, kSatElems << 8);   // bytes stay below 2^61
}

Costs tree_costs(const Analysis& an, const Program& prog, uint64_t k) {
    Costs c;
    for (int v = an.L; v < int(an.nodes.size()); ++v) {
        const Node& nd = an.nodes[v];
        const double unit = std::ldexp(1.0, nd.q + int(nd.legs.size()));
        c.C += double(nd.kv) * unit;
        c.single += double(k) * unit;
        c.RW += double(nd.kv) * (std::ldexp(1.0, int(an.nodes[nd.l].legs.size())) +
                                 std::ldexp(1.0, int(an.nodes[nd.r].legs.size())) +
                                 std::ldexp(1.0, int(nd.legs.size())));
    }
    c.perm = prog.permute_elems;
    return c;
}

namespace {
constexpr double kProfileBw = 6.6e12 * 0.6;  // bytes/s reached by streaming kernels
}

double contraction_time(double cmac, double bytes, bool tensor_core, int precision) {
    const double simt = precision == XEB_PREC_FP64 ? 0.3e12 : 10.0e12 * 0.5;  // complex MAC/s
    const double tc = 1.0e15 / 3.0 / 8.0 * 0.6;            // 3 TF32 products per complex MAC
    return std::max(cmac / (tensor_core ? tc : simt), bytes / kProfileBw) + 3e-6;
}

double expected_distinct(int b, uint64_t k) {
    if (b <= 0 || k == 0) return 1.0;
    if (b >= 60) return double(k);
    const double n = std::ldexp(1.0, b);
    return n * -std::expm1(double(k) * std::log1p(-1.0 / n));
}

double estimate_time(const Analysis& an, const Program& prog, int precision, size_t elem) {
    double t = 0;
    for (const Op& op : prog.ops) {
        if (op.kind == OP_PERM) {
            t += 2.0 * double(op.keys) * std::ldexp(1.0, op.r) * double(elem) / kProfileBw + 3e-6;
            continue;
        }
        const double cmac = double(op.kv) * double(op.M) * double(op.N) * double(op.K);
        const double bytes = double(elem) * (double(an.nodes[op.a_node].kv) * std::ldexp(1.0, op.a_rank) +
                                             double(an.nodes[op.b_node].kv) * std::ldexp(1.0, op.b_rank) +
                                             double(op.kv) * double(op.M) * double(op.N));
        t += contraction_time(cmac, bytes, precision == XEB_PREC_TF32X3 && tc_eligible(op), precision);
    }
    return t;
}

// ---- planners ---------------------------------------------------------------------

Tree greedy_tree(const Network& net, DistinctCounter& dc, const std::vector<int>& sliced,
                 uint64_t seed, double noise) {
    struct Item {
        int ref;
        std::vector<int> legs;  // sorted
        uint64_t mask;
        int64_t kv;
        bool alive;
    };
    std::set<int> sl(sliced.begin(), sliced.end());
    std::vector<Item> items;
    std::vector<std::vector<int>> owners(net.n_legs);
    for (size_t j = 0; j < net.leaves.size(); ++j) {
        Item it;
        it.ref = -1 - int(j);
        for (int l : net.leaves[j].legs)
            if (!sl.count(l)) it.legs.push_back(l);
        std::sort(it.legs.begin(), it.legs.end());
        it.mask = 0;
        for (int q : net.leaves[j].out_q) it.mask |= uint64_t(1) << q;
        it.kv = dc.count(it.mask);
        it.alive = true;
        for (int l : it.legs) owners[l].push_back(int(items.size()));
        items.push_back(std::move(it));
    }
    const bool exact = dc.k <= 20000;
    std::mt19937_64 rng(seed);
    std::normal_distribution<double> gauss(0.0, 1.0);
    Tree tree;
    int alive = int(items.size());
    auto sym = [](const std::vector<int>& a, const std::vector<int>& b) {
        std::vector<int> r;
        std::set_symmetric_difference(a.begin(), a.end(), b.begin(), b.end(), std::back_inserter(r));
        return r;
    };
    while (alive > 1) {
        double best = 0;
        int bi = -1, bj = -1;
        std::set<std::pair<int, int>> done;
        for (int l = 0; l < net.n_legs; ++l) {
            if (owners[l].size() != 2) continue;
            int i = owners[l][0], j = owners[l][1];
            if (i > j) std::swap(i, j);
            if (!done.insert({i, j}).second) continue;
            const Item& A = items[i];
            const Item& B = items[j];
            const std::vector<int> res = sym(A.legs, B.legs);
            const uint64_t m = A.mask | B.mask;
            const double kv = exact ? double(dc.count(m)) : std::min(double(A.kv) * double(B.kv), double(dc.k));
            double score = kv * std::ldexp(1.0, int(res.size())) - double(A.kv) * std::ldexp(1.0, int(A.legs.size())) -
                           double(B.kv) * std::ldexp(1.0, int(B.legs.size()));
            if (noise > 0) score += noise * std::fabs(score) * gauss(rng);
            if (bi < 0 || score < best) { best = score; bi = i; bj = j; }
        }
        if (bi < 0) {  // disconnected: outer product of the two smallest
            std::vector<int> al;
            for (size_t i = 0; i < items.size(); ++i)
                if (items[i].alive) al.push_back(int(i));
            std::sort(al.begin(), al.end(), [&](int x, int y) {
                return items[x].legs.size() < items[y].legs.size() ||
                       (items[x].legs.size() == items[y].legs.size() && x < y);
            });
            bi = std::min(al[0], al[1]);
            bj = std::max(al[0], al[1]);
        }
        Item M;
        M.legs = sym(items[bi].legs, items[bj].legs);
        M.mask = items[bi].mask | items[bj].mask;
        M.kv = dc.count(M.mask);
        M.alive = true;
        tree.push_back({items[bi].ref, items[bj].ref});
        M.ref = int(tree.size()) - 1;
        items[bi].alive = items[bj].alive = false;
        for (int l : items[bi].legs) owners[l].erase(std::remove(owners[l].begin(), owners[l].end(), bi), owners[l].end());
        for (int l : items[bj].legs) owners[l].erase(std::remove(owners[l].begin(), owners[l].end(), bj), owners[l].end());
        const int mi = int(items.size());
        for (int l : M.legs) owners[l].push_back(mi);
        items.push_back(std::move(M));
        --alive;
    }
    return tree;
}

// Frontier blocks over the body leaves (time order = leaf order).
static std::vector<std::vector<int>> frontier_blocks(const Network& net, const std::vector<int>& body, int bmax) {
    const int n = net.n;
    std::vector<std::vector<int>> per_q(n);  // body leaves on each qubit, time order
    for (int j : body)
        for (int q : net.leaves[j].qubits) per_q[q].push_back(j);
    std::vector<size_t> head(n, 0);
    std::vector<char> done(net.leaves.size(), 0);
    auto ready = [&](int j) {
        for (int q : net.leaves[j].qubits)
            if (head[q] >= per_q[q].size() || per_q[q][head[q]] != j) return false;
        return true;
    };
    auto absorb = [&](int j, std::vector<int>& blk) {
        done[j] = 1;
        blk.push_back(j);
        for (int q : net.leaves[j].qubits) ++head[q];
    };
    std::vector<std::vector<int>> blocks;
    size_t left = body.size();
    while (left > 0) {
        int first = -1;
        for (int j : body)
            if (!done[j] && ready(j)) { first = j; break; }
        if (first < 0) break;  // cannot happen for a circuit network
        std::set<int> Q(net.leaves[first].qubits.begin(), net.leaves[first].qubits.end());
        std::vector<int> blk;
        for (;;) {
            bool grew = false;
            for (int q : Q) {
                while (head[q] < per_q[q].size()) {
                    const int j = per_q[q][head[q]];
                    bool inside = ready(j);
                    for (int qq : net.leaves[j].qubits)
                        if (!Q.count(qq)) inside = false;
                    if (!inside) break;
                    absorb(j, blk);
                    grew = true;
                }
            }
            if (grew) continue;
            // widen the window by the earliest ready gate that still fits
            int best = -1;
            for (int q : Q) {
                if (head[q] >= per_q[q].size()) continue;
                const int j = per_q[q][head[q]];
                if (!ready(j)) continue;
                std::set<int> U = Q;
                U.insert(net.leaves[j].qubits.begin(), net.leaves[j].qubits.end());
                if (int(U.size()) <= bmax && (best < 0 || j < best)) best = j;
            }
            if (best < 0) {
                // no ready neighbour fits: take the earliest ready gate anywhere
                // that fits (disjoint gates then share one pass over the state)
                for (int j : body) {
                    if (done[j] || !ready(j)) continue;
                    std::set<int> U = Q;
                    U.insert(net.leaves[j].qubits.begin(), net.leaves[j].qubits.end());
                    if (int(U.size()) <= bmax) { best = j; break; }
                }
            }
            if (best < 0) break;
            Q.insert(net.leaves[best].qubits.begin(), net.leaves[best].qubits.end());
        }
        left -= blk.size();
        std::sort(blk.begin(), blk.end());
        blocks.push_back(blk);
    }
    return blocks;
}

bool sweep_tree(const Network& net, int bmax, int G, Tree& tree, int variant) {
    const int L = int(net.leaves.size());
    tree.clear();
    if (L < 2 || bmax < 2 || G < 1) return false;
    std::vector<int> outs, body;
    for (int j = 0; j < L; ++j) (net.leaves[j].out_q.empty() ? body : outs).push_back(j);
    // body blocks: gates grouped while their qubit set stays <= bmax
    struct Blk {
        std::set<int> qs;
        std::vector<int> leaves;
        int created;
    };
    std::vector<Blk> open;
    std::vector<std::vector<int>> closed;
    int created = 0;
    auto close_blk = [&](size_t i) {
        closed.push_back(open[i].leaves);
        open.erase(open.begin() + i);
    };
    for (int j : body) {
        const std::vector<int>& qs = net.leaves[j].qubits;
        std::vector<size_t> hit;
        for (size_t i = 0; i < open.size(); ++i)
            for (int q : qs)
                if (open[i].qs.count(q)) { hit.push_back(i); break; }
        std::set<int> U(qs.begin(), qs.end());
        for (size_t i : hit) U.insert(open[i].qs.begin(), open[i].qs.end());
        if (int(U.size()) <= bmax) {
            Blk nb;
            nb.qs = U;
            nb.created = created++;
            for (size_t i : hit) nb.leaves.insert(nb.leaves.end(), open[i].leaves.begin(), open[i].leaves.end());
            nb.leaves.push_back(j);
            std::sort(nb.leaves.begin(), nb.leaves.end());
            for (size_t t = hit.size(); t-- > 0;) open.erase(open.begin() + hit[t]);
            open.push_back(std::move(nb));
        } else {
            // close the blocks that hold these qubits, oldest first
            std::sort(hit.begin(), hit.end(), [&](size_t x, size_t y) { return open[x].created < open[y].created; });
            std::vector<int> ids;
            for (size_t i : hit) ids.push_back(open[i].created);
            for (int id : ids)
                for (size_t i = 0; i < open.size(); ++i)
                    if (open[i].created == id) { close_blk(i); break; }
            Blk nb;
            nb.qs = std::set<int>(qs.begin(), qs.end());
            nb.created = created++;
            nb.leaves = {j};
            open.push_back(std::move(nb));
        }
    }
    std::sort(open.begin(), open.end(), [](const Blk& x, const Blk& y) { return x.created < y.created; });
    for (auto& b : open) closed.push_back(b.leaves);
    if (variant == 1) closed = frontier_blocks(net, body, bmax);
    auto chain = [&](const std::vector<int>& lv) {
        int ref = -1 - lv[0];
        for (size_t t = 1; t < lv.size(); ++t) {
            tree.push_back({ref, -1 - lv[t]});
            ref = int(tree.size()) - 1;
        }
        return ref;
    };
    int spine = 0;
    bool have = false;
    for (auto& blk : closed) {
        const int r = chain(blk);
        if (!have) { spine = r; have = true; }
        else { tree.push_back({spine, r}); spine = int(tree.size()) - 1; }
    }
    for (size_t g = 0; g < outs.size(); g += size_t(G)) {
        std::vector<int> grp(outs.begin() + g, outs.begin() + std::min(outs.size(), g + size_t(G)));
        const int r = chain(grp);
        if (!have) { spine = r; have = true; }
        else { tree.push_back({spine, r}); spine = int(tree.size()) - 1; }
    }
    return int(tree.size()) == L - 1;
}

}  // namespace xebp
