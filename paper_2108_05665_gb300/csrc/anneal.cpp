// Local search over contraction trees and slice sets (App. A, "Contraction
// trees optimization" and "Slicing"): simulated annealing with the four
// associativity/commutativity rewrites, gains computed locally (App. C: a
// rewrite of (T1*T2)*T3 into T1*(T2*T3) changes only the cost of the new
// inner node and of the node above it), and slicing moves every K proposals.
#include "plan.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <random>
#include <thread>

namespace xebp {

namespace {

int popc(uint64_t x) { return __builtin_popcountll(x); }

struct Annealer {
    const Network& net;
    const uint64_t k;
    const AnnealOpts ao;
    int L = 0, N = 0, W = 0, root = -1;
    std::vector<std::array<int, 2>> ch;  // children of internal nodes (leaves: -1)
    std::vector<int> par;
    std::vector<uint64_t> base;          // leaf legs, all legs (L x W)
    std::vector<uint64_t> legs;          // node legs without sliced ones (N x W)
    std::vector<uint64_t> mask;          // output qubits below each node
    std::vector<double> kv, tv, gv;      // distinct keys, time term, memory term
    std::vector<char> sl;                // sliced legs
    int n_sliced = 0;
    double T = 0, Ms = 0;
    std::mt19937_64 rng;

    Annealer(const Network& n_, uint64_t k_, const AnnealOpts& a) : net(n_), k(k_), ao(a), rng(a.seed) {}

    uint64_t* lg(int v) { return legs.data() + size_t(v) * W; }
    const uint64_t* lg(int v) const { return legs.data() + size_t(v) * W; }

    double keys(uint64_t m) const { return m ? expected_distinct(popc(m), k) : 1.0; }

    // memory term of a node: (k_v 2^{r_v} / M_max)^p, capped so sums stay finite
    double gterm(double kvv, int r) const {
        const double l2 = std::log2(kvv) + r - std::log2(ao.budget_elems);
        return std::exp2(std::min(ao.p * l2, 1000.0));
    }

    // time of the contraction that forms a node from children with legs a, b
    double tterm(double kvv, double ka, double kb, const uint64_t* a, const uint64_t* b) const {
        int la = 0, lb = 0, lu = 0, lk = 0;
        for (int w = 0; w < W; ++w) {
            la += popc(a[w]);
            lb += popc(b[w]);
            lu += popc(a[w] | b[w]);
            lk += popc(a[w] & b[w]);
        }
        const int lv = lu - lk;
        const double cmac = kvv * std::ldexp(1.0, lu);
        const double bytes = double(ao.elem) * (ka * std::ldexp(1.0, la) + kb * std::ldexp(1.0, lb) +
                                                kvv * std::ldexp(1.0, lv));
        // the tensor-core form: one key, a free side of >= 128 rows, the other
        // free side and the summed side 16..64 wide
        const int fa = la - lk, fb = lb - lk;
        const bool tc = ao.precision == XEB_PREC_TF32X3 && kvv <= 1.0 && lk >= 4 && lk <= 6 &&
                        std::max(fa, fb) >= 7 && std::min(fa, fb) >= 4 && std::min(fa, fb) <= 6;
        return contraction_time(cmac, bytes, tc, ao.precision);
    }

    void init(const Tree& tree, const std::vector<int>& sliced) {
        L = int(net.leaves.size());
        N = 2 * L - 1;
        W = (net.n_legs + 63) / 64;
        ch.assign(N, {-1, -1});
        par.assign(N, -1);
        base.assign(size_t(L) * W, 0);
        legs.assign(size_t(N) * W, 0);
        mask.assign(N, 0);
        kv.assign(N, 1.0);
        tv.assign(N, 0.0);
        gv.assign(N, 0.0);
        for (int j = 0; j < L; ++j) {
            for (int l : net.leaves[j].legs) base[size_t(j) * W + l / 64] |= uint64_t(1) << (l % 64);
            for (int q : net.leaves[j].out_q) mask[j] |= uint64_t(1) << q;
        }
        auto id = [&](int ref) { return ref < 0 ? -1 - ref : L + ref; };
        for (int i = 0; i < L - 1; ++i) {
            const int v = L + i;
            ch[v] = {id(tree[i][0]), id(tree[i][1])};
            par[ch[v][0]] = par[ch[v][1]] = v;
        }
        root = L + (L - 2);
        sl.assign(net.n_legs, 0);
        n_sliced = 0;
        for (int l : sliced)
            if (!sl[l]) { sl[l] = 1; ++n_sliced; }
        recompute();
    }

    // post-order over internal nodes
    std::vector<int> order() const {
        std::vector<int> out, st{root};
        std::vector<char> seen(N, 0);
        while (!st.empty()) {
            const int v = st.back();
            if (v < L) { st.pop_back(); continue; }
            if (!seen[v]) {
                seen[v] = 1;
                st.push_back(ch[v][1]);
                st.push_back(ch[v][0]);
            } else {
                st.pop_back();
                out.push_back(v);
            }
        }
        return out;
    }

    void node_update(int v) {
        const int a = ch[v][0], b = ch[v][1];
        uint64_t* o = lg(v);
        for (int w = 0; w < W; ++w) o[w] = lg(a)[w] ^ lg(b)[w];
        mask[v] = mask[a] | mask[b];
        kv[v] = keys(mask[v]);
        int r = 0;
        for (int w = 0; w < W; ++w) r += popc(o[w]);
        gv[v] = gterm(kv[v], r);
        tv[v] = tterm(kv[v], kv[a], kv[b], lg(a), lg(b));
    }

    void recompute() {
        std::vector<uint64_t> slw(W, 0);
        for (int l = 0; l < net.n_legs; ++l)
            if (sl[l]) slw[l / 64] |= uint64_t(1) << (l % 64);
        for (int j = 0; j < L; ++j) {
            for (int w = 0; w < W; ++w) lg(j)[w] = base[size_t(j) * W + w] & ~slw[w];
            kv[j] = keys(mask[j]);
        }
        T = 0;
        Ms = 0;
        for (int v : order()) {
            node_update(v);
            T += tv[v];
            Ms += gv[v];
        }
    }

    double f_of(double t, double ms, int ns) const {
        const double m = 1.0 + std::log2(std::max(ms, 1e-300)) / ao.p;  // log2(2 (sum)^(1/p)) in budget units
        return ao.beta * std::max(m, 0.0) + double(ns) + std::log2(std::max(t, 1e-12));
    }
    double f() const { return f_of(T, Ms, n_sliced); }

    bool over_budget() const { return 1.0 + std::log2(std::max(Ms, 1e-300)) / ao.p > 0.0; }

    // One rewrite proposal at node v: its child X = (x0, x1) and the other
    // child Y; swap Y with x_i.  Returns true if accepted.
    bool propose(double temp) {
        std::uniform_int_distribution<int> pick(L, N - 1);
        const int v = pick(rng);
        const int s0 = int(rng() & 1);
        int s = s0;
        if (ch[v][s] < L) s ^= 1;
        if (ch[v][s] < L) return false;
        const int X = ch[v][s], Y = ch[v][s ^ 1];
        const int i = int(rng() & 1);
        const int xi = ch[X][i], xo = ch[X][i ^ 1];
        // candidate X' = (Y, xo), v = (X', xi)
        uint64_t nx[64];
        for (int w = 0; w < W; ++w) nx[w] = lg(Y)[w] ^ lg(xo)[w];
        const uint64_t nm = mask[Y] | mask[xo];
        const double nk = keys(nm);
        int r = 0;
        for (int w = 0; w < W; ++w) r += popc(nx[w]);
        const double ng = gterm(nk, r);
        const double ntx = tterm(nk, kv[Y], kv[xo], lg(Y), lg(xo));
        const double ntv = tterm(kv[v], nk, kv[xi], nx, lg(xi));
        double T2 = T - tv[X] - tv[v] + ntx + ntv;
        double M2 = Ms - gv[X] + ng;
        // a removed term that dominates the sum: recompute it instead of
        // subtracting (no cancellation)
        if (tv[X] + tv[v] > 0.25 * T) {
            T2 = ntx + ntv;
            for (int u = L; u < N; ++u)
                if (u != X && u != v) T2 += tv[u];
        }
        if (gv[X] > 0.25 * Ms) {
            M2 = ng;
            for (int u = L; u < N; ++u)
                if (u != X) M2 += gv[u];
        }
        const double d = f_of(T2, M2, n_sliced) - f();
        if (d > 0) {
            std::uniform_real_distribution<double> U(0.0, 1.0);
            if (temp <= 0 || U(rng) >= std::exp(-d / temp)) return false;
        }
        ch[X] = {Y, xo};
        ch[v][s] = X;
        ch[v][s ^ 1] = xi;
        par[Y] = X;
        par[xi] = v;
        for (int w = 0; w < W; ++w) lg(X)[w] = nx[w];
        mask[X] = nm;
        kv[X] = nk;
        gv[X] = ng;
        tv[X] = ntx;
        tv[v] = ntv;
        T = T2;
        Ms = M2;
        return true;
    }

    // Slicing move (App. A, "Slicing"): over budget, add the leg of the
    // largest tensors whose slicing gives the smallest memory estimate (ties:
    // smaller f); otherwise drop the sliced leg whose removal gives the
    // smallest f, if that lowers f (the paper drops a random one; trying each
    // keeps the search from accumulating legs a rewritten tree no longer needs).
    void slice_move() {
        if (over_budget() && n_sliced < ao.max_sliced) {
            double mx = 0;
            for (int v = L; v < N; ++v) mx = std::max(mx, gv[v]);
            std::vector<char> cand(net.n_legs, 0);
            for (int v = L; v < N; ++v)
                if (gv[v] * std::exp2(ao.p) >= mx)
                    for (int w = 0; w < W; ++w)
                        for (uint64_t x = lg(v)[w]; x; x &= x - 1) cand[w * 64 + __builtin_ctzll(x)] = 1;
            int bl = -1;
            double bm = 0, bf = 0;
            for (int l = 0; l < net.n_legs; ++l) {
                if (!cand[l] || net.is_open_leg(l)) continue;
                sl[l] = 1;
                ++n_sliced;
                recompute();
                const double m = Ms, ff = f();
                sl[l] = 0;
                --n_sliced;
                if (bl < 0 || m < bm * (1 - 1e-9) || (m <= bm * (1 + 1e-9) && ff < bf)) {
                    bl = l;
                    bm = m;
                    bf = ff;
                }
            }
            if (bl >= 0) {
                sl[bl] = 1;
                ++n_sliced;
            }
            recompute();
        } else if (n_sliced > 0) {
            const double f0 = f();
            int bl = -1;
            double bf = f0;
            for (int l = 0; l < net.n_legs; ++l) {
                if (!sl[l]) continue;
                sl[l] = 0;
                --n_sliced;
                recompute();
                const double ff = f();
                sl[l] = 1;
                ++n_sliced;
                if (ff < bf - 1e-12) {
                    bf = ff;
                    bl = l;
                }
            }
            if (bl >= 0) {
                sl[bl] = 0;
                --n_sliced;
            }
            recompute();
        }
    }

    Tree tree() const {
        Tree t;
        std::vector<int> ref(N, 0);
        for (int j = 0; j < L; ++j) ref[j] = -1 - j;
        for (int v : order()) {
            t.push_back({ref[ch[v][0]], ref[ch[v][1]]});
            ref[v] = int(t.size()) - 1;
        }
        return t;
    }

    std::vector<int> sliced() const {
        std::vector<int> s;
        for (int l = 0; l < net.n_legs; ++l)
            if (sl[l]) s.push_back(l);
        return s;
    }
};

}  // namespace

void anneal_tree(const Network& net, uint64_t k, Tree& tree, std::vector<int>& sliced, const AnnealOpts& ao,
                 AnnealStats* stats) {
    const int L = int(net.leaves.size());
    if (L < 3 || ao.steps <= 0 || (net.n_legs + 63) / 64 > 64) return;
    Annealer a(net, k, ao);
    a.init(tree, sliced);
    double best_f = a.f();
    if (stats) stats->f_start = best_f;
    Tree best_t = tree;
    std::vector<int> best_s = a.sliced();
    int64_t acc = 0;
    const double ratio = ao.t1 / ao.t0;
    const int64_t refresh = std::max<int64_t>(1, 50 * int64_t(L));
    for (int64_t step = 0; step < ao.steps; ++step) {
        const double temp = ao.t0 * std::pow(ratio, double(step) / double(ao.steps));
        if (a.propose(temp)) ++acc;
        if (ao.slice_every > 0 && (step + 1) % ao.slice_every == 0) a.slice_move();
        else if ((step + 1) % refresh == 0) a.recompute();  // drop rounding drift of the running sums
        const double f = a.f();
        if (f < best_f - 1e-12) {
            // the running sums drift; confirm a new best on fresh sums
            a.recompute();
            const double fr = a.f();
            if (fr < best_f - 1e-12) {
                best_f = fr;
                best_t = a.tree();
                best_s = a.sliced();
            }
        }
    }
    tree = best_t;
    sliced = best_s;
    if (stats) {
        stats->f_best = best_f;
        stats->accepted = acc;
    }
}

void anneal_many(const Network& net, uint64_t k, std::vector<Tree>& trees, std::vector<std::vector<int>>& sliced,
                 const AnnealOpts& ao, std::vector<AnnealStats>& stats) {
    const size_t n = trees.size();
    stats.assign(n, AnnealStats());
    if (sliced.size() != n) sliced.resize(n);
    std::atomic<size_t> next(0);
    auto work = [&]() {
        for (size_t i; (i = next.fetch_add(1)) < n;) {
            AnnealOpts a = ao;
            a.seed = ao.seed * 7919 + i;
            anneal_tree(net, k, trees[i], sliced[i], a, &stats[i]);
        }
    };
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const size_t nt = std::min<size_t>(n, hw);
    std::vector<std::thread> th;
    for (size_t t = 1; t < nt; ++t) th.emplace_back(work);
    work();
    for (auto& t : th) t.join();
}

}  // namespace xebp
