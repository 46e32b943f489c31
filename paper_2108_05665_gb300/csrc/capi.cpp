// C ABI (include/xeb.h): planning, device layout of a plan, and the driver
// that enqueues the kernels of kernels.cu in tree order.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <memory>
#include <string>
#include <unordered_map>
#include <vector>

#include "kernels.cuh"
#include "plan.h"
#include "xeb.h"

using namespace xebp;

namespace {
thread_local std::string g_err;

xeb_status fail(xeb_status s, const std::string& msg) {
    g_err = msg;
    return s;
}
}  // namespace

void xebp::set_last_error(const std::string& msg) { g_err = msg; }

namespace {

#define XEB_CUDA(call)                                                                       \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail(XEB_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));      \
    } while (0)

int64_t align_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

constexpr int GK_TC2 = 101;  // tcgen05 split-precision kernel, W^T in tensor memory (tc_gemm2.cu)
constexpr int GK_TCKD = 102; // tcgen05 split-precision kernel for deep-K keyed contractions (tc_kdeep.cu)
// Defaults of the split-precision options (xeb_plan_opts.split_bits,
// split_terms, timeout_ms): big parts of 10 bits on a common grid, four
// products, 2 s per device-side wait.  With 11 bits the big*big sums of the
// 30-qubit workload pass 2^24 grid units often enough to bias F by 1.3e-6;
// with three products the missing small*small term (2^-20 of the grid)
// costs 1.7e-5 per amplitude.
constexpr int kSplitBitsDefault = 10;
constexpr int kSplitTermsDefault = 4;
constexpr uint32_t kTimeoutMsDefault = 2000;

// kernel-form choices of a contraction (autotuner candidates)
// (CH_STREAM_N2 / CH_STREAM_HALF: tile shapes of the streaming kernel -- two
// result columns per thread, so a warp stores whole result rows; half the
// rows per tile)
enum Choice {
    CH_AUTO = -1, CH_TC2 = 0, CH_TC2_GATHER = 1, CH_GROUPED = 2, CH_TCKD = 3, CH_SIMT = 4, CH_KEYED = 5, CH_KEYED2 = 6,
    CH_STREAM_N2 = 7, CH_STREAM_HALF = 8, CH_COUNT = 9
};

struct GemmLaunch {
    CUtensorMap tmap;  // A of a TMA-mode tensor-core launch (64-byte aligned)
    int kernel;
    xebk::GemmDesc d;
    xebk::StreamDesc s;
    xebk::TcDesc tc;
    xebk::KdDesc kd;
    int64_t kvB = 1;   // GK_KEYED: distinct right operands (keys of B's node)
    int rpt = 1;       // GK_KEYED: rows per lane (1 or 2)
};

// Result bits below this C address bit are kept inside one tensor-core tile,
// so every 32-byte sector of C is written whole by a single tile.
constexpr int kTileLowCBits = 3;

// Tensor-core eligibility and descriptor of a contraction (one key, 128-row
// tiles, 16 <= K, N <= 64 complex, tile offsets within 32 bits).
bool tc_tile(const Op& op, xebk::TcDesc& t, int row_bits, bool tmem_variant) {
    if (!tc_eligible(op)) return false;
    if (op.a_pos_m.size() > size_t(xebk::kMaxLegs)) return false;
    std::memset(&t, 0, sizeof(t));
    t.M = op.M;
    t.K2 = int(2 * op.K);
    t.N2 = int(2 * op.N);
    t.n_chunks = t.K2 / 32;
    t.tmem_cols = 4 * t.N2;  // 2 buffers x (big, small) accumulators
    // rows of a tile: for the tensor-memory kernel the rows whose output bits
    // are below kTileLowCBits come first so every tile writes whole sectors;
    // then the lowest remaining rows
    std::vector<int> tile_rows;
    if (tmem_variant) {
        for (size_t i = 0; i < op.a_pos_m.size(); ++i)
            if (op.c_pos_m[i] < kTileLowCBits) tile_rows.push_back(int(i));
        for (size_t i = 0; i < op.a_pos_m.size() && int(tile_rows.size()) < row_bits; ++i)
            if (std::find(tile_rows.begin(), tile_rows.end(), int(i)) == tile_rows.end()) tile_rows.push_back(int(i));
        if (int(tile_rows.size()) != row_bits) return false;
        std::sort(tile_rows.begin(), tile_rows.end());
    } else {
        for (int i = 0; i < row_bits; ++i) tile_rows.push_back(i);
        // the shared-memory variant writes row-major results only
        for (size_t i = 0; i < op.c_pos_m.size(); ++i)
            if (op.c_pos_m[i] != int(op.c_pos_n.size() + i)) return false;
    }
    std::vector<std::pair<int, int>> bits;
    for (int i : tile_rows) bits.push_back({op.a_pos_m[i], 0});
    for (int i = 0; i < 4; ++i) bits.push_back({op.a_pos_k[i], 1});
    std::sort(bits.begin(), bits.end());
    for (auto& b : bits)
        if (b.first > 30) return false;
    t.T = int(bits.size());
    for (int i = 0; i < t.T; ++i) {
        t.pos[i] = int8_t(bits[i].first);
        if (bits[i].second) t.is_k |= 1u << i;
    }
    for (int c = 0; c < t.n_chunks; ++c) {
        int64_t o = 0;
        for (size_t i = 4; i < op.a_pos_k.size(); ++i)
            if ((c >> (i - 4)) & 1) o |= int64_t(1) << op.a_pos_k[i];
        if (o > INT32_MAX) return false;
        t.chunk_off[c] = int32_t(o);
    }
    t.nam = int(op.a_pos_m.size());
    for (int i = 0; i < t.nam; ++i) t.apm[i] = int8_t(op.a_pos_m[i]);
    t.n_ext = 0;
    for (int i = 0; i < t.nam; ++i) {
        if (std::find(tile_rows.begin(), tile_rows.end(), i) != tile_rows.end()) continue;
        t.ext_apos[t.n_ext] = int8_t(op.a_pos_m[i]);
        t.ext_cpos[t.n_ext] = int8_t(op.c_pos_m[i]);
        ++t.n_ext;
    }
    std::vector<std::array<int, 3>> st;  // (C bit, is column, bit index)
    for (size_t r = 0; r < tile_rows.size(); ++r) st.push_back({op.c_pos_m[tile_rows[r]], 0, int(r)});
    for (size_t j = 0; j < op.c_pos_n.size(); ++j) st.push_back({op.c_pos_n[j], 1, int(j)});
    std::sort(st.begin(), st.end());
    if (st.size() > 16) return false;
    t.Tst = int(st.size());
    t.st_is_n = 0;
    for (int i = 0; i < t.Tst; ++i) {
        t.st_pos[i] = int8_t(st[i][0]);
        t.st_idx[i] = int8_t(st[i][2]);
        if (st[i][1]) t.st_is_n |= 1u << i;
    }
    // Staging swizzle: the epilogue reads the tile with lane bit i = tile bit
    // i (i < 5) of ascending C order, 8 bytes per lane; the bank pair of slot
    // row * 64 + n' is n' mod 16.  Column bits j < 4 move it by 2^j; row bits
    // and column bits >= 4 do not, so each of those lane bits gets an unused
    // unit vector of GF(2)^4: the 16 lanes of a half-warp then read 16
    // distinct bank pairs (no conflicts) whatever the result layout.
    std::memset(t.st_swz, 0, sizeof(t.st_swz));
    if (tmem_variant) {
        unsigned used = 0;
        for (int i = 0; i < 4 && i < t.Tst; ++i)
            if (st[i][1] && st[i][2] < 4) used |= 1u << st[i][2];
        for (int i = 0; i < 4 && i < t.Tst; ++i) {
            if (st[i][1] && st[i][2] < 4) continue;
            int m = 0;
            while (m < 4 && ((used >> m) & 1)) ++m;
            if (m == 4) break;
            used |= 1u << m;
            t.st_swz[i] = int8_t(1 << m);
        }
    }
    t.nbk = int(op.b_pos_k.size());
    t.nbn = int(op.b_pos_n.size());
    for (int i = 0; i < t.nbk; ++i) t.bpk[i] = int8_t(op.b_pos_k[i]);
    for (int i = 0; i < t.nbn; ++i) t.bpn[i] = int8_t(op.b_pos_n[i]);
    // TMA mode (candidate; the tensor map is encoded at bind): A is a
    // row-major [M][K] matrix and the tile's lowest >= 3 row bits are the
    // matrix's lowest rows, so a tile is 16 boxes of 8 consecutive whole rows
    t.tma = 0;
    if (tmem_variant && op.M <= (int64_t(1) << 31)) {
        const int nak = int(op.a_pos_k.size());
        bool row_major = true;
        for (int i = 0; i < nak; ++i) row_major = row_major && op.a_pos_k[i] == i;
        for (size_t i = 0; i < op.a_pos_m.size(); ++i) row_major = row_major && op.a_pos_m[i] == nak + int(i);
        int a = 0;
        while (a < row_bits && tile_rows[a] == a) ++a;
        if (row_major && a >= 3) {
            t.tma = 1;
            a = 3;
            t.box_log2 = a;
            t.row_shift = nak;
            for (int j = 0; j < (1 << (row_bits - a)); ++j) {
                int64_t y = 0;
                for (int b = 0; b < row_bits - a; ++b)
                    if ((j >> b) & 1) y |= int64_t(1) << tile_rows[a + b];
                t.box_y[j] = int32_t(y);
            }
        }
    }
    return true;
}

// Grouped tensor-core form of a memo-level contraction (N = 1, keys grouped
// by their left key): each group is a GEMM whose columns are the group's keys,
// their B vectors packed contiguously by the memo prep kernel.  Possible when
// groups are long (>= 512 tiles) and hold at most 64 keys; opt-in, because
// with K = 16 a tile is one 32 KB chunk and the kernel's per-tile hand-offs
// cost more than the SIMT memo-level kernel's arithmetic.
bool tc_grouped(const Analysis& an, const Op& op, const xebk::GemmDesc& d, xebk::TcDesc& t) {
    if (op.N != 1 || op.kv <= 1 || !d.gstart || !d.c_natural) return false;
    if (op.M < (int64_t(1) << 16) || op.K < 16 || op.K > 64) return false;
    const int64_t kvB = an.nodes[op.b_node].kv;
    if (kvB > 64 || d.c_key != op.M) return false;
    int64_t npad = 16;
    while (npad < kvB) npad *= 2;
    int lk = 0, ln = 0, lm = 0;
    while ((int64_t(1) << lk) < op.K) ++lk;
    while ((int64_t(1) << ln) < npad) ++ln;
    while ((int64_t(1) << lm) < op.M) ++lm;
    Op o2 = op;
    o2.kv = 1;
    o2.N = npad;
    o2.b_pos_k.clear();
    o2.b_pos_n.clear();
    o2.c_pos_m.clear();
    o2.c_pos_n.clear();
    for (int i = 0; i < lk; ++i) o2.b_pos_k.push_back(i);
    for (int i = 0; i < ln; ++i) o2.b_pos_n.push_back(lk + i);
    for (int i = 0; i < lm; ++i) o2.c_pos_m.push_back(i);
    for (int i = 0; i < ln; ++i) o2.c_pos_n.push_back(lm + i);
    o2.c_hint.clear();
    if (!tc_tile(o2, t, xebk::kTc2RowBits, true)) return false;
    t.tma = 0;
    t.grp = 1;
    std::memset(t.st_swz, 0, sizeof(t.st_swz));
    t.tpg = op.M >> xebk::kTc2RowBits;
    t.n_groups = d.n_groups;
    t.c_key = d.c_key;
    t.gstart = d.gstart;
    return true;
}

// Deep-K keyed tensor-core form (tc_kdeep.cu): C_u = A_uL(u) (M x K)
// B_uR(u) (K x N), M, N in {16, 32}, K >= 64 a multiple of 64 complex: many
// keys of a deep sum with small results.
bool tc_kdeep(const Op& op, const xebk::GemmDesc& d, xebk::KdDesc& k) {
    auto small = [](int64_t x) { return x == 16 || x == 32; };
    if (op.kv < 2 || !d.uL || !d.uR || !small(op.M) || !small(op.N) || op.K < 64 || op.K % 64 != 0 || op.K > 8192)
        return false;
    if (d.nak != d.nbk || d.nak > xebk::kMaxLegs || d.nam > 5 || d.nbn > 5) return false;
    std::memset(&k, 0, sizeof(k));
    k.a_off = d.a_off;
    k.a_key = d.a_key;
    k.b_off = d.b_off;
    k.b_key = d.b_key;
    k.c_off = d.c_off;
    k.c_key = d.c_key;
    k.uL = d.uL;
    k.uR = d.uR;
    k.gstart = d.gstart;
    k.n_groups = d.n_groups;
    k.kv = op.kv;
    k.M = int(op.M);
    k.N = int(op.N);
    k.K = int(op.K);
    k.nak = d.nak;
    k.nbk = d.nbk;
    for (int i = 0; i < d.nam; ++i) {
        k.apm[i] = d.apm[i];
        k.cpm[i] = d.cpm[i];
    }
    for (int i = 0; i < d.nbn; ++i) {
        k.bpn[i] = d.bpn[i];
        k.cpn[i] = d.cpn[i];
    }
    for (int i = 0; i < d.nak; ++i) {
        k.apk[i] = d.apk[i];
        k.bpk[i] = d.bpk[i];
    }
    return true;
}

// Keyed tensor-core form: C_u = A_uL(u) B_uR(u) for every key u with the
// single-key tile rules (128-row tiles, 16 <= K, N <= 64), one group of
// M / 128 tiles per key; gathered A rows, W^T of the key's B written into
// tensor memory when a CTA's tiles move to the next key.
bool tc_keyed(const Op& op, const xebk::GemmDesc& d, xebk::TcDesc& t) {
    if (op.kv <= 1 || op.M < 128 || op.M % 128 != 0 || op.K < 16 || op.K > 64 || op.N < 16 || op.N > 64) return false;
    Op o1 = op;
    o1.kv = 1;
    if (!tc_tile(o1, t, xebk::kTc2RowBits, true)) return false;
    t.tma = 0;
    t.grp = 1;
    t.keyed = 1;
    t.tpg = op.M >> xebk::kTc2RowBits;
    t.n_groups = op.kv;
    t.c_key = d.c_key;
    t.a_key = d.a_key;
    t.b_key = d.b_key;
    t.uL = d.uL;
    t.uR = d.uR;
    t.gstart = nullptr;
    return true;
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled_fn() {
    static EncodeTiledFn fn = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return EncodeTiledFn(nullptr);
        return reinterpret_cast<EncodeTiledFn>(f);
    }();
    return fn;
}

// Tensor map of a TMA-mode launch's A operand: the row-major [M rows][2K
// floats] matrix seen as (32 floats of a chunk, row, chunk), boxes of 32
// floats x 2^box_log2 rows x all 2K/32 chunks, 128-byte swizzle: one box is
// 2^box_log2 whole rows, laid out chunk-major in shared memory.
// False (the launch then gathers with plain loads) if the base is not 16-byte
// aligned or the driver refuses the map.
bool encode_a_map(const xebk::TcDesc& t, const float2* arena, CUtensorMap& map) {
    const float2* base = arena + t.a_off;
    if (reinterpret_cast<uintptr_t>(base) % 16 != 0) return false;
    EncodeTiledFn fn = encode_tiled_fn();
    if (!fn) return false;
    const cuuint64_t dims[3] = {32u, cuuint64_t(t.M), cuuint64_t(t.n_chunks)};
    const cuuint64_t strides[2] = {cuuint64_t(t.K2) * 4, 128u};
    const cuuint32_t box[3] = {32u, cuuint32_t(1u << t.box_log2), cuuint32_t(t.n_chunks)};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    return fn(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float2*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Tile shape of the streaming kernel for a contraction, or false if the
// contraction does not fit it.
// npt_force > 0: that many result columns per thread (a divisor of N);
// half_rows: half the rows per tile the default rule picks.
bool stream_tile(const Op& op, size_t elem, xebk::StreamDesc& s, int npt_force = 0, bool half_rows = false) {
    if (op.K > xebk::kStreamMaxK || op.N > xebk::kStreamMaxN || op.M < 64) return false;
    int npt = op.N <= 8 ? int(op.N) : (op.N == 16 ? 8 : 16);
    if (npt_force > 0) {
        if (op.N < npt_force || op.N % npt_force != 0) return false;
        npt = npt_force;
    }
    const int tpr = int(op.N) >= npt ? int(op.N) / npt : 1;
    const int rg = 256 / tpr;
    int R = 1;
    while (2 * R <= op.M && 2 * R * op.K <= 256 * xebk::kStreamEPT && 2 * R <= rg * std::max(1, 16 / npt) &&
           size_t(2 * R) * size_t(op.K) * elem <= 16 * 1024)
        R *= 2;
    if (half_rows) R /= 2;
    if (R < 32 || R * op.K > 256 * xebk::kStreamEPT) return false;
    int tm = 0;
    while ((1 << tm) < R) ++tm;
    for (int q : op.a_pos_k)
        if (q > 30) return false;  // tile offsets are 32-bit
    for (int i = 0; i < tm; ++i)
        if (op.a_pos_m[i] > 30) return false;
    // tile bits: the tm lowest row bits and all summed bits, ascending address
    std::vector<std::pair<int, int>> bits;  // (address position, is_k)
    for (int i = 0; i < tm; ++i) bits.push_back({op.a_pos_m[i], 0});
    for (int p : op.a_pos_k) bits.push_back({p, 1});
    std::sort(bits.begin(), bits.end());
    if (bits.size() > 32) return false;
    s.R = R;
    s.tm = tm;
    s.T = int(bits.size());
    s.npt = npt;
    s.is_k = 0;
    for (int i = 0; i < s.T; ++i) {
        s.pos[i] = int8_t(bits[i].first);
        if (bits[i].second) s.is_k |= 1u << i;
    }
    return true;
}
}  // namespace

struct xeb_plan_s {
    Network net;
    int w = 0;               // open qubits (multi-batch): 2^w amplitudes per bitstring
    xebk::RootMap rootmap{};  // where open-qubit bit j sits in the root's per-key block
    // cross-slice reuse: a node is contracted in a slice only if a slice bit
    // in node_mask[v] changed since the previous slice (all ones: always)
    std::vector<uint32_t> node_mask;
    int n_reused = 0;         // nodes whose result is kept across slices
    // constant folding: subtrees that depend on no output bit, no sliced leg
    // and no open leg are evaluated once on the host in FP64 (fold_roots: the
    // largest such subtrees, their values in the root node's stored layout);
    // their leaves and contractions never run on the device
    int test_wait = 0;                 // xeb_plan_test_wait
    std::vector<char> folded;          // per node: inside a folded subtree
    std::vector<char> op_folded;       // per program op
    std::vector<int> fold_roots;
    std::vector<std::vector<cd>> fold_vals;
    Tree tree;
    std::vector<int> sliced;
    Analysis an;
    Program prog;
    Costs costs;
    double objective = 0;
    int planner_used = 0;
    xeb_plan_opts opts{};
    std::vector<uint64_t> bits;
    size_t k = 0;
    size_t elem = 8;
    // device state
    bool bound = false;
    bool owns = false;
    char* ws = nullptr;
    size_t ws_bytes = 0;
    int64_t off_arena = 0, off_leafdata = 0, off_tables = 0;
    size_t bytes_total = 0;
    // offsets inside tables (bytes)
    int64_t t_trie_desc = 0, t_internal = 0, t_leaf_desc = 0, t_pi = 0, t_bits = 0, t_acc = 0, t_amps = 0,
            t_partials = 0, t_result = 0, t_err = 0, t_sort = 0, t_memo = 0;
    size_t memo_bytes = 0;
    std::vector<int> choice;   // per op: CH_AUTO or the autotuner's form
    bool slice_all = true;           // the loop runs every slice value in counting order
    std::vector<int64_t> slice_ids;  // else these slice values, in this order (possibly none)
    int n_sms = 152;
    int64_t tables_bytes = 0;
    std::vector<xebk::TrieDesc> trie;
    std::vector<int> trie_of_node;  // node -> index in trie, -1 if no bits
    std::vector<int> trie_internal;
    std::vector<xebk::LeafDesc> leafdesc;   // leaves materialised on the device
    std::vector<int> leafdesc_leaf;         // ... their leaf ids
    std::vector<int64_t> leaf_src_off;
    int64_t leafdata_elems = 0;
    std::vector<xebk::PermDesc> perms;  // per op (unused for GEMM)
    std::vector<GemmLaunch> gemms;      // per op (unused for PERM)
    int max_kv = 1;
    int n_xeb_blocks = 64;
    bool tables_ready = false;
    bool amps_ready = false;
    // profiling
    bool profiling = false;
    struct Rec {
        int cls;
        cudaEvent_t a, b;
        double flops, bytes;
        int op;  // program op index, -1 for non-contraction kernels
    };
    std::vector<Rec> pending;
    // A whole step (key tables + every slice + XEB) as one CUDA graph,
    // captured on a private stream and launched on the caller's stream.  A
    // profiled graph also holds an event-record node before and after every
    // kernel; its events are read before the graph is launched again, so two
    // profiled graphs alternate and the host never waits on the step in flight.
    struct StepGraph {
        cudaGraphExec_t exec = nullptr;
        void* out = nullptr;
        std::vector<Rec> recs;
        bool launched = false;
    };
    cudaStream_t cap_stream = nullptr;
    StepGraph graph_plain, graph_prof[2];
    int graph_prof_next = 0;
    bool capturing_prof = false;
    std::vector<cudaEvent_t> event_pool;
    double prof_ms[XEB_N_KC] = {0}, prof_n[XEB_N_KC] = {0}, prof_flops[XEB_N_KC] = {0}, prof_bytes[XEB_N_KC] = {0};
    std::vector<double> op_ms, op_n;  // per program op
};

namespace {
cudaEvent_t take_event(xeb_plan_s* p) {
    if (!p->event_pool.empty()) {
        cudaEvent_t e = p->event_pool.back();
        p->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Brackets one launch with events when profiling is on.
struct ProfScope {
    xeb_plan_s* p;
    cudaStream_t st;
    int cls;
    double flops, bytes;
    int op;
    cudaEvent_t a = nullptr;
    ProfScope(xeb_plan_s* p_, cudaStream_t st_, int cls_, double flops_, double bytes_, int op_ = -1)
        : p(p_), st(st_), cls(cls_), flops(flops_), bytes(bytes_), op(op_) {
        if (p->profiling) {
            a = take_event(p);
            record(a);
        }
    }
    void record(cudaEvent_t e) {
        // inside a capture an external record becomes an event-record node
        if (p->capturing_prof)
            cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
        else
            cudaEventRecord(e, st);
    }
    ~ProfScope() {
        if (!p->profiling || !a) return;
        cudaEvent_t b = take_event(p);
        record(b);
        p->pending.push_back({cls, a, b, flops, bytes, op});
    }
};

void accumulate(xeb_plan_s* p, const std::vector<xeb_plan_s::Rec>& recs) {
    for (const auto& r : recs) {
        float ms = 0.f;
        if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            p->prof_ms[r.cls] += ms;
            p->prof_n[r.cls] += 1;
            p->prof_flops[r.cls] += r.flops;
            p->prof_bytes[r.cls] += r.bytes;
            if (r.op >= 0) {
                if (p->op_ms.size() <= size_t(r.op)) {
                    p->op_ms.resize(size_t(r.op) + 1, 0.0);
                    p->op_n.resize(size_t(r.op) + 1, 0.0);
                }
                p->op_ms[size_t(r.op)] += ms;
                p->op_n[size_t(r.op)] += 1;
            }
        }
    }
}

void drain_profile(xeb_plan_s* p) {
    accumulate(p, p->pending);
    for (auto& r : p->pending) {
        p->event_pool.push_back(r.a);
        p->event_pool.push_back(r.b);
    }
    p->pending.clear();
    for (auto& g : p->graph_prof)
        if (g.launched) {
            accumulate(p, g.recs);
            g.launched = false;
        }
}

void drop_graph(xeb_plan_s* p, xeb_plan_s::StepGraph& g) {
    if (g.launched) accumulate(p, g.recs);
    if (g.exec) cudaGraphExecDestroy(g.exec);
    for (auto& r : g.recs) {
        p->event_pool.push_back(r.a);
        p->event_pool.push_back(r.b);
    }
    g = xeb_plan_s::StepGraph();
}
}  // namespace

extern "C" {

const char* xeb_last_error(void) { return g_err.c_str(); }

void xeb_default_opts(xeb_plan_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = XEB_PREC_FP32;
    o->planner = XEB_PLANNER_AUTO;
    o->beta = 10.0;
    o->mem_budget = uint64_t(64) << 30;
    o->seed = 1;
    o->greedy_trials = 4;
}

xeb_status xeb_network_info(const xeb_circuit* c, int* n_leaves, int* n_legs) {
    Network net;
    std::string err;
    if (!build_network(c, net, err)) return fail(XEB_EINVAL, err);
    if (n_leaves) *n_leaves = int(net.leaves.size());
    if (n_legs) *n_legs = net.n_legs;
    return XEB_OK;
}

xeb_status xeb_network_leaves(const xeb_circuit* c, int32_t* out_bits, int32_t* legs) {
    Network net;
    std::string err;
    if (!build_network(c, net, err)) return fail(XEB_EINVAL, err);
    for (size_t j = 0; j < net.leaves.size(); ++j) {
        const Leaf& lf = net.leaves[j];
        if (out_bits)
            for (int t = 0; t < 2; ++t) out_bits[2 * j + t] = t < int(lf.out_q.size()) ? lf.out_q[t] : -1;
        if (legs)
            for (int t = 0; t < 4; ++t) legs[4 * j + t] = t < int(lf.legs.size()) ? lf.legs[t] : -1;
    }
    return XEB_OK;
}

}  // extern "C"

namespace {

struct Candidate {
    Tree tree;
    Analysis an;
    Program prog;
    Costs costs;
    double f = 0;
    int64_t arena_bytes = 0;
};

bool evaluate(const Network& net, const Tree& tree, const std::vector<int>& sliced, DistinctCounter& dc,
              const xeb_plan_opts& o, size_t elem, uint64_t k, Candidate& cand, std::string& err,
              bool orient = true) {
    cand.tree = tree;
    if (orient && check_tree(tree, int(net.leaves.size()), err)) orient_tree(net, cand.tree, sliced);
    const Tree& tree_ = cand.tree;
    if (!analyze(net, tree_, sliced, cand.an, err)) return false;
    fill_counts(cand.an, dc);
    build_program(cand.an, cand.prog, o.reserved[0] == 0, o.precision == XEB_PREC_TF32X3);
    plan_memory(cand.prog);
    cand.costs = tree_costs(cand.an, cand.prog, k);
    cand.arena_bytes = cand.prog.arena_elems * int64_t(elem);
    const double budget = double(std::max<uint64_t>(o.mem_budget, 1));
    const double nsl = std::ldexp(1.0, int(sliced.size()));
    const double mem_term = o.beta * std::max(std::log2(double(cand.arena_bytes) / budget), 0.0);
    if (o.alpha > 0) {
        // App. A objective with arithmetic intensity alpha
        cand.f = mem_term + std::log2(nsl * (cand.costs.C + o.alpha * (cand.costs.RW + cand.costs.perm)) + 1.0);
    } else {
        // efficiency-profile variant: log2 of the estimated time (seconds)
        cand.f = mem_term + std::log2(nsl * estimate_time(cand.an, cand.prog, o.precision, elem));
    }
    return true;
}

// Slicing (App. A, "Slicing"): while the arena exceeds the budget, add the
// leg that minimises the objective f (memory penalty + log2 of the total
// time over all slices); ties go to the smaller arena, then the smaller
// largest tensor, then the smaller total tensor size.
void slice_candidate(const Network& net, DistinctCounter& dc, const xeb_plan_opts& o, size_t elem, uint64_t k,
                     Candidate& best, std::vector<int>& sliced, std::string& err, bool orient = true) {
        auto node_elems = [](const Analysis& an, int v) {
            return double(an.nodes[v].kv) * std::ldexp(1.0, int(an.nodes[v].legs.size()));
        };
        auto measure = [&](const Candidate& c) {
            double mx = 0, tot = 0;
            for (size_t v = 0; v < c.an.nodes.size(); ++v) {
                const double e = node_elems(c.an, int(v));
                mx = std::max(mx, e);
                tot += e;
            }
            return std::array<double, 4>{c.f, double(c.arena_bytes), mx, tot};
        };
        while (uint64_t(best.arena_bytes) > o.mem_budget && sliced.size() < 30) {
            const auto mb = measure(best);
            std::vector<int> legs;
            for (size_t v = 0; v < best.an.nodes.size(); ++v)
                if (node_elems(best.an, int(v)) * 2 >= mb[2])
                    for (int l : best.an.nodes[v].legs)
                        if (std::find(legs.begin(), legs.end(), l) == legs.end()) legs.push_back(l);
            Candidate bc;
            std::array<double, 4> bm{};
            int bl = -1;
            for (int l : legs) {
                std::vector<int> s2 = sliced;
                s2.push_back(l);
                Candidate c;
                if (!evaluate(net, best.tree, s2, dc, o, elem, k, c, err, orient)) continue;
                const auto m = measure(c);
                if (bl < 0 || m < bm) {
                    bc = std::move(c);
                    bm = m;
                    bl = l;
                }
            }
            if (bl < 0 || !(bm < mb)) break;
            sliced.push_back(bl);
            best = std::move(bc);
        }
    }

// The planner's candidate trees: randomised greedy restarts and the sweep
// family (body blocks of b qubits, output leaves in groups of G, two variants).
std::vector<std::pair<int, Tree>> candidate_trees(const Network& net, DistinctCounter& dc,
                                                  const std::vector<int>& sliced, const xeb_plan_opts& o) {
    std::vector<std::pair<int, Tree>> cands;
        if (o.planner == XEB_PLANNER_AUTO || o.planner == XEB_PLANNER_ANNEAL || o.planner == XEB_PLANNER_GREEDY) {
            const int trials = std::max(1, o.greedy_trials);
            for (int t = 0; t < trials; ++t)
                cands.push_back({XEB_PLANNER_GREEDY, greedy_tree(net, dc, sliced, o.seed + t, t == 0 ? 0.0 : 0.15)});
        }
        if (o.planner == XEB_PLANNER_AUTO || o.planner == XEB_PLANNER_ANNEAL || o.planner == XEB_PLANNER_SWEEP) {
            std::vector<int> bs, gs;
            if (o.block_qubits > 0) bs = {o.block_qubits};
            else for (int b = 2; b <= 10; ++b) bs.push_back(b);
            if (o.group_leaves > 0) gs = {o.group_leaves};
            else gs = {1, 2, 3, 4};
            for (int variant = 0; variant < 2; ++variant)
                for (int b : bs)
                    for (int g : gs) {
                        Tree t;
                        if (sweep_tree(net, b, g, t, variant)) cands.push_back({XEB_PLANNER_SWEEP, t});
                    }
        }
    return cands;
}

// Plan features of the learned cost model (XEB_N_FEATURES values): exact
// counter totals over all slices, the hand time model, and per kernel class
// (as the default kernel selection assigns them: tensor core, streaming,
// memo level, tiled, small) the count, bytes and flops of its contractions.
void plan_features(const Candidate& c, size_t n_sliced, const xeb_plan_opts& o, size_t elem, uint64_t k, int n,
                   double* f) {
    for (int i = 0; i < XEB_N_FEATURES; ++i) f[i] = 0;
    auto lg = [](double x) { return std::log2(1.0 + std::max(0.0, x)); };
    const double nsl = std::ldexp(1.0, int(n_sliced));
    const bool tf32 = o.precision == XEB_PREC_TF32X3;
    double cls_n[5] = {0}, cls_b[5] = {0}, cls_f[5] = {0};
    double tot_b = 0, tot_f = 0, b_k4 = 0, b_n4 = 0, b_small_m = 0, max_e = 0, max_kv = 0, tot_e = 0;
    for (const Op& op : c.prog.ops) {
        if (op.kind == OP_PERM) continue;
        const double fl = 8.0 * double(op.kv) * double(op.M) * double(op.N) * double(op.K);
        const double by = double(elem) * (double(c.an.nodes[op.a_node].kv) * double(op.M) * double(op.K) +
                                          double(c.an.nodes[op.b_node].kv) * double(op.K) * double(op.N) +
                                          double(op.kv) * double(op.M) * double(op.N));
        xebk::StreamDesc sd;
        int cl;
        if (tf32 && tc_eligible(op)) cl = 0;
        else if (stream_tile(op, elem, sd)) cl = (op.N == 1 && op.kv > 1) ? 2 : 1;
        else if (op.N > 1 && op.M >= 16 && op.N >= 16) cl = 3;
        else cl = 4;
        cls_n[cl] += 1;
        cls_b[cl] += by;
        cls_f[cl] += fl;
        tot_b += by;
        tot_f += fl;
        if (op.K <= 4) b_k4 += by;
        if (op.N <= 4) b_n4 += by;
        if (op.M < 4096) b_small_m += by;
    }
    for (const auto& nd : c.an.nodes) {
        const double e = double(nd.kv) * std::ldexp(1.0, int(nd.legs.size()));
        max_e = std::max(max_e, e);
        max_kv = std::max(max_kv, double(nd.kv));
        tot_e += e;
    }
    f[0] = lg(c.costs.C * nsl);
    f[1] = lg(c.costs.RW * nsl);
    f[2] = lg(c.costs.perm * nsl);
    f[3] = double(n_sliced);
    f[4] = lg(double(c.arena_bytes));
    f[5] = lg(1e6 * nsl * estimate_time(c.an, c.prog, o.precision, elem));
    f[6] = lg(double(c.prog.ops.size()));
    f[7] = lg(double(k));
    f[8] = double(n);
    for (int cl = 0; cl < 5; ++cl) {
        f[9 + 3 * cl] = lg(cls_n[cl] * nsl);
        f[10 + 3 * cl] = lg(cls_b[cl] * nsl);
        f[11 + 3 * cl] = lg(cls_f[cl] * nsl);
    }
    f[24] = lg(max_e);
    f[25] = lg(max_kv);
    f[26] = tot_b > 0 ? b_k4 / tot_b : 0;
    f[27] = tot_b > 0 ? b_n4 / tot_b : 0;
    f[28] = lg(tot_e * nsl);
    f[29] = tf32 ? 1.0 : 0.0;
    f[30] = tot_f > 0 ? cls_f[0] / tot_f : 0;
    f[31] = lg(b_small_m * nsl);
}

}  // namespace

namespace {
// Cross-slice reuse.  A node's tensor depends on the slice value only through
// the sliced legs of its subtree (m_v, a mask of slice bits).  Going down from
// the root, a child keeps its own mask where it is strictly smaller than its
// parent's effective mask e (so it can be skipped while the parent is
// recomputed, and its buffer stays reserved for the whole step), else takes
// the parent's (it is recomputed with the parent, its buffer lives as usual).
// In slice t a node is contracted iff t = 0 or (s_t ^ s_{t-1}) & e_v != 0.
// Off when the reserved buffers would push the arena above the plan's budget
// (or above its own arena if that is larger), in permute-first mode, or with
// opts.reserved[7] = 1.
void setup_reuse(xeb_plan_s* p) {
    const Analysis& an = p->an;
    const int N = int(an.nodes.size()), L = an.L, S = int(p->sliced.size());
    const uint32_t all = S >= 32 ? ~0u : (1u << S) - 1;
    p->node_mask.assign(size_t(N), ~0u);
    p->n_reused = 0;
    if (S == 0 || p->opts.reserved[7] == 1 || p->opts.reserved[0] == 1) return;
    std::vector<uint32_t> m(size_t(N), 0);
    for (int j = 0; j < L; ++j)
        for (int l : p->net.leaves[size_t(j)].legs) {
            const auto it = std::find(p->sliced.begin(), p->sliced.end(), l);
            if (it != p->sliced.end()) m[size_t(j)] |= 1u << int(it - p->sliced.begin());
        }
    for (int v = L; v < N; ++v) m[size_t(v)] = m[size_t(an.nodes[size_t(v)].l)] | m[size_t(an.nodes[size_t(v)].r)];
    std::vector<uint32_t> e(size_t(N), all);
    std::vector<int> keep;
    for (int v = N - 1; v >= L; --v)
        for (int c : {an.nodes[size_t(v)].l, an.nodes[size_t(v)].r}) {
            if (m[size_t(c)] != e[size_t(v)] && c >= L) {
                e[size_t(c)] = m[size_t(c)];
                keep.push_back(c);
            } else {
                e[size_t(c)] = e[size_t(v)];
            }
        }
    if (keep.empty()) return;
    Program pr = p->prog;
    for (int c : keep) {
        Buffer& b = pr.bufs[size_t(pr.node_buf[size_t(c)])];
        b.first = 0;
        b.last = int(pr.ops.size()) + 1;
    }
    plan_memory(pr);
    const double cap = std::max(double(p->opts.mem_budget), double(p->prog.arena_elems) * double(p->elem));
    if (double(pr.arena_elems) * double(p->elem) > cap) return;
    p->prog = std::move(pr);
    for (int v = 0; v < N; ++v) p->node_mask[size_t(v)] = e[size_t(v)];
    p->n_reused = int(keep.size());
}

// Host FP64 tensor: legs slowest first, element index bit (size-1-i) = leg i.
struct HostT {
    std::vector<int> legs;
    std::vector<cd> t;
};

// Pairwise contraction (Eq. elem-cont) of two host tensors over their shared
// legs; result legs: a's unshared legs, then b's.
HostT host_contract(const HostT& a, const HostT& b) {
    std::vector<int> sh, fa, fb;
    for (int l : a.legs)
        (std::find(b.legs.begin(), b.legs.end(), l) != b.legs.end() ? sh : fa).push_back(l);
    for (int l : b.legs)
        if (std::find(sh.begin(), sh.end(), l) == sh.end()) fb.push_back(l);
    auto bit_of = [](const std::vector<int>& lay, int leg) {
        return int(lay.size()) - 1 - int(std::find(lay.begin(), lay.end(), leg) - lay.begin());
    };
    HostT r;
    r.legs = fa;
    r.legs.insert(r.legs.end(), fb.begin(), fb.end());
    const int no = int(r.legs.size()), ns = int(sh.size());
    std::vector<int64_t> oa(no, 0), ob(no, 0), sa(ns), sb(ns);
    for (int i = 0; i < no; ++i) {
        const int leg = r.legs[i];
        const bool in_a = i < int(fa.size());
        (in_a ? oa : ob)[no - 1 - i] = int64_t(1) << bit_of(in_a ? a.legs : b.legs, leg);
    }
    for (int j = 0; j < ns; ++j) {
        sa[j] = int64_t(1) << bit_of(a.legs, sh[j]);
        sb[j] = int64_t(1) << bit_of(b.legs, sh[j]);
    }
    r.t.assign(size_t(1) << no, cd(0, 0));
    for (int64_t o = 0; o < (int64_t(1) << no); ++o) {
        int64_t ia = 0, ib = 0;
        for (int i = 0; i < no; ++i)
            if ((o >> i) & 1) { ia += oa[i]; ib += ob[i]; }
        cd acc(0, 0);
        for (int64_t u = 0; u < (int64_t(1) << ns); ++u) {
            int64_t ja = ia, jb = ib;
            for (int j = 0; j < ns; ++j)
                if ((u >> j) & 1) { ja += sa[j]; jb += sb[j]; }
            acc += a.t[size_t(ja)] * b.t[size_t(jb)];
        }
        r.t[size_t(o)] = acc;
    }
    return r;
}

// Constant folding (see xeb_plan_s::folded).  A node qualifies when its
// subtree depends on no output bit, sliced leg or open leg and every tensor in
// it has at most max_legs legs; the qualifying internal nodes whose parent
// does not qualify are evaluated on the host and their buffers reserved for
// the whole step.  Off in permute-first mode.
void fold_constants(xeb_plan_s* p) {
    const Analysis& an = p->an;
    const int N = int(an.nodes.size()), L = an.L;
    p->folded.assign(size_t(N), 0);
    p->op_folded.assign(p->prog.ops.size(), 0);
    p->fold_roots.clear();
    p->fold_vals.clear();
    const int max_legs = p->opts.fold_legs == 0 ? 16 : p->opts.fold_legs;
    if (max_legs < 0 || p->opts.reserved[0] == 1) return;
    std::vector<char> ok(size_t(N), 0);
    for (int v = 0; v < N; ++v) {
        const Node& nd = an.nodes[size_t(v)];
        bool q = nd.qmask == 0 && int(nd.legs.size()) <= max_legs && nd.q + int(nd.legs.size()) <= 24;
        if (v < L) {
            for (int l : p->net.leaves[size_t(v)].legs)
                q = q && !p->net.is_open_leg(l) &&
                    std::find(p->sliced.begin(), p->sliced.end(), l) == p->sliced.end();
            q = q && p->net.leaves[size_t(v)].out_q.empty();
        } else {
            q = q && ok[size_t(nd.l)] && ok[size_t(nd.r)];
        }
        ok[size_t(v)] = q;
    }
    std::vector<HostT> val(static_cast<size_t>(N));
    for (int v = L; v < N - 1; ++v) {
        const Node& nd = an.nodes[size_t(v)];
        if (!ok[size_t(v)] || ok[size_t(nd.parent)]) continue;
        // evaluate the subtree of v in post-order (children have smaller ids)
        std::vector<int> sub, stack{v};
        while (!stack.empty()) {
            const int u = stack.back();
            stack.pop_back();
            sub.push_back(u);
            p->folded[size_t(u)] = 1;
            if (u >= L) {
                stack.push_back(an.nodes[size_t(u)].l);
                stack.push_back(an.nodes[size_t(u)].r);
            }
        }
        std::sort(sub.begin(), sub.end());
        for (int u : sub) {
            if (u < L) {
                val[size_t(u)].legs = p->net.leaves[size_t(u)].legs;
                val[size_t(u)].t = p->net.leaves[size_t(u)].t;
            } else {
                val[size_t(u)] = host_contract(val[size_t(an.nodes[size_t(u)].l)], val[size_t(an.nodes[size_t(u)].r)]);
                val[size_t(an.nodes[size_t(u)].l)] = HostT();
                val[size_t(an.nodes[size_t(u)].r)] = HostT();
            }
        }
        // values in the stored layout of v's result
        const HostT& h = val[size_t(v)];
        const std::vector<int>& lay = p->prog.layout[size_t(v)];
        const int r = int(lay.size());
        std::vector<int64_t> inc(static_cast<size_t>(r));
        for (int i = 0; i < r; ++i) {
            const int at = int(std::find(h.legs.begin(), h.legs.end(), lay[size_t(i)]) - h.legs.begin());
            inc[size_t(r - 1 - i)] = int64_t(1) << (int(h.legs.size()) - 1 - at);
        }
        std::vector<cd> out(size_t(1) << r);
        for (int64_t x = 0; x < (int64_t(1) << r); ++x) {
            int64_t src = 0;
            for (int i = 0; i < r; ++i)
                if ((x >> i) & 1) src += inc[size_t(i)];
            out[size_t(x)] = h.t[size_t(src)];
        }
        val[size_t(v)] = HostT();
        p->fold_roots.push_back(v);
        p->fold_vals.push_back(std::move(out));
        Buffer& b = p->prog.bufs[size_t(p->prog.node_buf[size_t(v)])];
        b.first = 0;
        b.last = int(p->prog.ops.size()) + 1;
    }
    if (p->fold_roots.empty()) return;
    for (size_t i = 0; i < p->prog.ops.size(); ++i)
        p->op_folded[i] = p->prog.ops[i].kind == OP_GEMM && p->folded[size_t(p->prog.ops[i].node)];
    plan_memory(p->prog);
}

xeb_status create_plan(const xeb_circuit* circuit, const uint64_t* bitstrings, size_t k, uint64_t open_mask,
                       const xeb_tree* tree, const xeb_slices* slices, const xeb_plan_opts* opts, xeb_plan_s** out) {
    if (!out) return fail(XEB_EINVAL, "out is NULL");
    *out = nullptr;
    if (k == 0 || !bitstrings) return fail(XEB_EINVAL, "need k >= 1 bitstrings");
    if (k > size_t(xebk::kMaxK))
        return fail(XEB_EUNSUPPORTED, "k > " + std::to_string(xebk::kMaxK) + " bitstrings per plan");
    std::unique_ptr<xeb_plan_s> p(new xeb_plan_s());
    if (opts) p->opts = *opts;
    else xeb_default_opts(&p->opts);
    const xeb_plan_opts& o = p->opts;
    if (o.precision != XEB_PREC_FP32 && o.precision != XEB_PREC_FP64 && o.precision != XEB_PREC_TF32X3)
        return fail(XEB_EINVAL, "unknown precision");
    if (o.split_bits != 0 && (o.split_bits < 8 || o.split_bits > 11))
        return fail(XEB_EINVAL, "split_bits must be 0 (default) or 8..11");
    if (o.split_terms != 0 && o.split_terms != 3 && o.split_terms != 4)
        return fail(XEB_EINVAL, "split_terms must be 0 (default), 3 or 4");
    if (o.timeout_ms > 600000) return fail(XEB_EINVAL, "timeout_ms above 600000 (ten minutes)");
    p->elem = o.precision == XEB_PREC_FP64 ? 16 : 8;
    std::string err;
    if (!build_network(circuit, p->net, err, open_mask)) return fail(XEB_EINVAL, err);
    p->w = p->net.n_open;
    if (p->w > 16) return fail(XEB_EUNSUPPORTED, "more than 16 open qubits");
    if (p->w == p->net.n) return fail(XEB_EUNSUPPORTED, "every qubit open: nothing to memoize (use a state vector)");
    const int n = p->net.n;
    for (size_t i = 0; i < k; ++i)
        if (n < 64 && (bitstrings[i] >> n) != 0) return fail(XEB_EINVAL, "bitstring has bits above n");
    p->bits.assign(bitstrings, bitstrings + k);
    p->k = k;
    DistinctCounter dc;
    dc.bs = p->bits.data();
    dc.k = k;
    if (slices && slices->n > 0) {
        if (!slices->legs) return fail(XEB_EINVAL, "slices->legs is NULL");
        p->sliced.assign(slices->legs, slices->legs + slices->n);
        if (p->sliced.size() > 30) return fail(XEB_EUNSUPPORTED, "more than 30 sliced legs");
    }
    Candidate best;
    bool have = false;
    std::vector<std::pair<double, Tree>> ranked;  // constructed trees by objective
    if (tree) {
        if (!tree->children && tree->n_nodes > 0) return fail(XEB_EINVAL, "tree->children is NULL");
        Tree t(tree->n_nodes);
        for (int i = 0; i < tree->n_nodes; ++i) t[i] = {tree->children[2 * i], tree->children[2 * i + 1]};
        if (!evaluate(p->net, t, p->sliced, dc, o, p->elem, k, best, err, false)) return fail(XEB_EINVAL, err);
        have = true;
        p->planner_used = 0;
    } else {
        if (p->net.leaves.size() < 2) return fail(XEB_EUNSUPPORTED, "network with fewer than two leaves");
        std::vector<std::pair<int, Tree>> cands = candidate_trees(p->net, dc, p->sliced, o);
        for (auto& c : cands) {
            Candidate cd_;
            if (!evaluate(p->net, c.second, p->sliced, dc, o, p->elem, k, cd_, err)) continue;
            ranked.push_back({cd_.f, c.second});
            if (!have || cd_.f < best.f) {
                best = std::move(cd_);
                have = true;
                p->planner_used = c.first;
            }
        }
        if (!have) return fail(XEB_EINVAL, "planner found no valid tree: " + err);
    }
    if (!slices) slice_candidate(p->net, dc, o, p->elem, k, best, p->sliced, err, tree == nullptr);
    // App. A local search: always for XEB_PLANNER_ANNEAL; under AUTO when the
    // constructed trees needed slicing to fit the budget or still do not fit.
    // Restarts begin from the best constructed trees and from randomised
    // greedy trees; the best few by the search's own objective are evaluated
    // exactly (distinct counts, emulated arena) and the best kept.
    if (!tree && (o.planner == XEB_PLANNER_ANNEAL ||
                  (o.planner == XEB_PLANNER_AUTO && !slices &&
                   (!p->sliced.empty() || uint64_t(best.arena_bytes) > o.mem_budget)))) {
        const int L = int(p->net.leaves.size());
        const int R = 16;
        std::sort(ranked.begin(), ranked.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
        std::vector<Tree> starts;
        for (size_t i = 0; i < ranked.size() && starts.size() < 4; ++i) starts.push_back(ranked[i].second);
        for (int r = int(starts.size()); r < R; ++r)
            starts.push_back(greedy_tree(p->net, dc, {}, o.seed + 1000 + uint64_t(r), 0.15));
        std::vector<std::vector<int>> sls(starts.size(), slices ? p->sliced : std::vector<int>());
        AnnealOpts ao;
        ao.steps = o.reserved[5] > 0 ? int64_t(o.reserved[5]) * 1000
                                     : std::min<int64_t>(int64_t(20) << 20, int64_t(100000) * L);
        ao.slice_every = slices ? 0 : std::max<int64_t>(1, ao.steps / 400);
        ao.t0 = 2.0;
        ao.t1 = 0.001;
        ao.beta = o.beta;
        ao.budget_elems = double(std::max<uint64_t>(o.mem_budget, 1)) / double(p->elem);
        ao.precision = o.precision;
        ao.elem = p->elem;
        ao.seed = o.seed;
        std::vector<AnnealStats> ast;
        anneal_many(p->net, k, starts, sls, ao, ast);
        std::vector<size_t> idx(starts.size());
        for (size_t i = 0; i < idx.size(); ++i) idx[i] = i;
        std::sort(idx.begin(), idx.end(), [&](size_t x, size_t y) {
            return ast[x].f_best < ast[y].f_best || (ast[x].f_best == ast[y].f_best && x < y);
        });
        bool took = false;
        for (size_t t = 0; t < std::min<size_t>(3, idx.size()); ++t) {
            std::vector<int> s = sls[idx[t]];
            Candidate c;
            if (!evaluate(p->net, starts[idx[t]], s, dc, o, p->elem, k, c, err)) continue;
            if (!slices) slice_candidate(p->net, dc, o, p->elem, k, c, s, err);
            if (c.f < best.f || (o.planner == XEB_PLANNER_ANNEAL && !took)) {
                best = std::move(c);
                p->sliced = s;
                p->planner_used = XEB_PLANNER_ANNEAL;
                took = true;
            }
        }
    }
    p->tree = best.tree;
    p->an = std::move(best.an);
    p->prog = std::move(best.prog);
    p->costs = best.costs;
    p->objective = best.f;
    {   // the root's block: its legs are exactly the open legs
        const std::vector<int>& lay = p->prog.layout[p->an.nodes.size() - 1];
        if (int(lay.size()) != p->w) return fail(XEB_EINVAL, "internal: root legs differ from the open legs");
        p->rootmap.w = p->w;
        for (int j = 0; j < p->w; ++j) {
            const int at = int(std::find(lay.begin(), lay.end(), p->net.open_legs[size_t(j)]) - lay.begin());
            p->rootmap.pos[j] = int8_t(int(lay.size()) - 1 - at);
        }
    }
    fold_constants(p.get());
    setup_reuse(p.get());
    *out = p.release();
    return XEB_OK;
}
}  // namespace

extern "C" xeb_status xeb_plan_create(const xeb_circuit* circuit, const uint64_t* bitstrings, size_t k,
                                      const xeb_tree* tree, const xeb_slices* slices,
                                      const xeb_plan_opts* opts, xeb_plan_s** out) {
    return create_plan(circuit, bitstrings, k, 0, tree, slices, opts, out);
}

extern "C" xeb_status xeb_plan_create_batched(const xeb_circuit* circuit, const uint64_t* bitstrings, size_t k,
                                              uint64_t open_mask, const xeb_tree* tree, const xeb_slices* slices,
                                              const xeb_plan_opts* opts, xeb_plan_s** out) {
    return create_plan(circuit, bitstrings, k, open_mask, tree, slices, opts, out);
}

extern "C" xeb_status xeb_plan_candidates(const xeb_circuit* circuit, const uint64_t* bitstrings, size_t k,
                                          const xeb_plan_opts* opts, int max_cands, int32_t* trees,
                                          int32_t* slices, int32_t* n_sliced, double* features, int32_t* planner,
                                          int32_t* n_out) {
    if (!n_out) return fail(XEB_EINVAL, "n_out is NULL");
    *n_out = 0;
    if (k == 0 || !bitstrings) return fail(XEB_EINVAL, "need k >= 1 bitstrings");
    if (k > size_t(xebk::kMaxK)) return fail(XEB_EUNSUPPORTED, "too many bitstrings");
    xeb_plan_opts o;
    if (opts) o = *opts;
    else xeb_default_opts(&o);
    const size_t elem = o.precision == XEB_PREC_FP64 ? 16 : 8;
    Network net;
    std::string err;
    if (!build_network(circuit, net, err)) return fail(XEB_EINVAL, err);
    if (net.leaves.size() < 2) return fail(XEB_EUNSUPPORTED, "network with fewer than two leaves");
    std::vector<uint64_t> bits(bitstrings, bitstrings + k);
    for (uint64_t b : bits)
        if (net.n < 64 && (b >> net.n) != 0) return fail(XEB_EINVAL, "bitstring has bits above n");
    DistinctCounter dc;
    dc.bs = bits.data();
    dc.k = k;
    const std::vector<int> none;
    const auto cands = candidate_trees(net, dc, none, o);
    const int nn = int(net.leaves.size()) - 1;
    int w = 0;
    for (const auto& c : cands) {
        if (w >= max_cands) break;
        Candidate cd;
        if (!evaluate(net, c.second, none, dc, o, elem, k, cd, err)) continue;
        std::vector<int> sl;
        slice_candidate(net, dc, o, elem, k, cd, sl, err);
        if (trees)
            for (int i = 0; i < nn; ++i) {
                trees[(size_t(w) * nn + i) * 2] = cd.tree[i][0];
                trees[(size_t(w) * nn + i) * 2 + 1] = cd.tree[i][1];
            }
        if (slices)
            for (int i = 0; i < 30; ++i) slices[size_t(w) * 30 + i] = i < int(sl.size()) ? sl[i] : -1;
        if (n_sliced) n_sliced[w] = int(sl.size());
        if (planner) planner[w] = c.first;
        if (features) plan_features(cd, sl.size(), o, elem, k, net.n, features + size_t(w) * XEB_N_FEATURES);
        ++w;
    }
    *n_out = w;
    return XEB_OK;
}

extern "C" xeb_status xeb_plan_create_learned(const xeb_circuit* circuit, const uint64_t* bitstrings, size_t k,
                                              const xeb_plan_opts* opts, xeb_mlp_s* model, int max_cands,
                                              uintptr_t stream, double* predicted_log2_ms, xeb_plan_s** out) {
    if (!circuit || !bitstrings || !model || !out) return fail(XEB_EINVAL, "NULL circuit, bitstrings, model or out");
    if (max_cands < 1) return fail(XEB_EINVAL, "max_cands < 1");
    if (predicted_log2_ms) *predicted_log2_ms = std::nan("");
    Network net;
    std::string err;
    if (!build_network(circuit, net, err)) return fail(XEB_EINVAL, err);
    if (net.leaves.size() < 2) return fail(XEB_EUNSUPPORTED, "network with fewer than two leaves");
    const int nn = int(net.leaves.size()) - 1;
    std::vector<int32_t> trees(size_t(max_cands) * size_t(nn) * 2), slices(size_t(max_cands) * 30), nsl(max_cands),
        fam(max_cands);
    std::vector<double> feat(size_t(max_cands) * XEB_N_FEATURES);
    int32_t n = 0;
    xeb_status s = xeb_plan_candidates(circuit, bitstrings, k, opts, max_cands, trees.data(), slices.data(),
                                       nsl.data(), feat.data(), fam.data(), &n);
    if (s != XEB_OK) return s;
    if (n == 0) return xeb_plan_create(circuit, bitstrings, k, nullptr, nullptr, opts, out);
    // predictions of log2 ms on the device
    std::vector<float> xf(static_cast<size_t>(n) * XEB_N_FEATURES), yf(static_cast<size_t>(n));
    for (size_t i = 0; i < xf.size(); ++i) xf[i] = float(feat[i]);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    float* xd = nullptr;
    float* yd = nullptr;
    cudaError_t e = cudaMalloc(&xd, xf.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&yd, yf.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpyAsync(xd, xf.data(), xf.size() * sizeof(float), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        s = xeb_mlp_forward(model, xd, n, yd, stream);
        if (s == XEB_OK) {
            e = cudaMemcpyAsync(yf.data(), yd, yf.size() * sizeof(float), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        }
    }
    if (xd) cudaFree(xd);
    if (yd) cudaFree(yd);
    if (s != XEB_OK) return s;
    if (e != cudaSuccess) return fail(XEB_ECUDA, std::string("learned planner: ") + cudaGetErrorString(e));
    int best = 0;
    for (int i = 1; i < n; ++i)
        if (yf[size_t(i)] < yf[size_t(best)]) best = i;
    if (predicted_log2_ms) *predicted_log2_ms = double(yf[size_t(best)]);
    const xeb_tree tree{nn, trees.data() + size_t(best) * size_t(nn) * 2};
    const xeb_slices sl{nsl[size_t(best)], slices.data() + size_t(best) * 30};
    return xeb_plan_create(circuit, bitstrings, k, &tree, nsl[size_t(best)] > 0 ? &sl : nullptr, opts, out);
}

extern "C" void xeb_plan_destroy(xeb_plan_s* p) {
    if (!p) return;
    drop_graph(p, p->graph_plain);
    for (auto& g : p->graph_prof) drop_graph(p, g);
    if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
    drain_profile(p);
    for (cudaEvent_t e : p->event_pool) cudaEventDestroy(e);
    if (p->owns && p->ws) cudaFree(p->ws);
    delete p;
}

extern "C" xeb_status xeb_plan_stats(xeb_plan_s* p, xeb_stats* s) {
    if (!p || !s) return fail(XEB_EINVAL, "NULL argument");
    std::memset(s, 0, sizeof(*s));
    s->n_qubits = p->net.n;
    s->n_leaves = int(p->net.leaves.size());
    s->n_legs = p->net.n_legs;
    s->n_nodes = int(p->tree.size());
    s->n_sliced = int(p->sliced.size());
    s->k = p->k;
    s->k_distinct = uint64_t(p->an.nodes.back().kv);
    s->flops_per_slice = 8.0 * p->costs.C;
    s->single_amp_flops = 8.0 * p->costs.single;
    s->rw_elems_per_slice = p->costs.RW;
    s->permute_elems_per_slice = p->costs.perm;
    s->objective = p->objective;
    s->arena_bytes = uint64_t(p->prog.arena_elems) * p->elem;
    s->device_bytes = xeb_plan_device_bytes(p);
    s->n_slices = uint64_t(1) << p->sliced.size();
    for (const Op& op : p->prog.ops) {
        if (op.kind == OP_GEMM) ++s->n_gemm_ops;
        else ++s->n_permute_ops;
    }
    s->planner_used = p->planner_used;
    s->reserved[0] = p->n_reused;
    for (char f : p->folded) s->reserved[1] += f != 0;
    s->reserved[2] = int(p->fold_roots.size());
    for (size_t i = 0; i < p->gemms.size() && i < p->prog.ops.size(); ++i)
        if (const GemmLaunch& g = p->gemms[i];
            p->prog.ops[i].kind != OP_PERM && !p->op_folded[i] && g.kernel == GK_TC2) {
            ++s->n_tc_launches;
            s->n_tc_tma += g.tc.tma != 0;
        }
    return XEB_OK;
}

extern "C" xeb_status xeb_plan_tree(xeb_plan_s* p, int32_t* children, int32_t* sliced_legs) {
    if (!p) return fail(XEB_EINVAL, "NULL plan");
    if (children)
        for (size_t i = 0; i < p->tree.size(); ++i) {
            children[2 * i] = p->tree[i][0];
            children[2 * i + 1] = p->tree[i][1];
        }
    if (sliced_legs)
        for (size_t i = 0; i < p->sliced.size(); ++i) sliced_legs[i] = p->sliced[i];
    return XEB_OK;
}

extern "C" xeb_status xeb_plan_node(xeb_plan_s* p, int node, int64_t* kv, int32_t* a, int32_t* b, int32_t* n_legs,
                                    int32_t* n_shared) {
    if (!p) return fail(XEB_EINVAL, "NULL plan");
    if (node < 0 || node >= int(p->tree.size())) return fail(XEB_EINVAL, "node out of range");
    const Node& nd = p->an.nodes[p->an.L + node];
    if (kv) *kv = nd.kv;
    if (a) *a = nd.a;
    if (b) *b = nd.b;
    if (n_legs) *n_legs = int32_t(nd.legs.size());
    if (n_shared) *n_shared = nd.q;
    return XEB_OK;
}

namespace {

// Device layout of a plan: [arena][leaf data][tables].
void layout_device(xeb_plan_s* p) {
    const Analysis& an = p->an;
    const int N = int(an.nodes.size());
    const int L = an.L;
    const int64_t A = 256;
    int64_t off = 0;
    p->off_arena = 0;
    off = align_up(p->prog.arena_elems * int64_t(p->elem), A);
    p->off_leafdata = off;
    p->leaf_src_off.assign(L, 0);
    int64_t le = 0;
    for (int j = 0; j < L; ++j) {
        p->leaf_src_off[j] = le;
        const Leaf& lf = p->net.leaves[j];
        le += int64_t(1) << (lf.out_q.size() + lf.legs.size());
    }
    p->leafdata_elems = le;
    off = align_up(off + le * int64_t(p->elem), A);
    p->off_tables = off;
    // tables
    int64_t t = 0;
    auto take = [&](int64_t bytes) {
        const int64_t r = t;
        t = align_up(t + std::max<int64_t>(bytes, 1), A);
        return r;
    };
    p->trie.clear();
    p->trie_of_node.assign(N, -1);
    p->trie_internal.clear();
    p->max_kv = 1;
    for (int v = 0; v < N; ++v)
        if (an.nodes[v].b > an.nodes[v].a) {
            p->trie_of_node[v] = int(p->trie.size());
            xebk::TrieDesc d{};
            d.a = an.nodes[v].a;
            d.b = an.nodes[v].b;
            d.kv = int(an.nodes[v].kv);
            d.is_internal = v >= L;
            p->trie.push_back(d);
            p->max_kv = std::max(p->max_kv, d.kv);
        }
    p->t_trie_desc = take(int64_t(p->trie.size()) * int64_t(sizeof(xebk::TrieDesc)));
    p->t_internal = take(int64_t(p->trie.size()) * 4);
    p->t_leaf_desc = take(int64_t(L) * int64_t(sizeof(xebk::LeafDesc)));
    p->t_pi = take(int64_t(p->net.n) * 4);
    p->t_bits = take(int64_t(p->k) * 8);
    for (int v = 0; v < N; ++v) {
        const int ti = p->trie_of_node[v];
        if (ti < 0) continue;
        xebk::TrieDesc& d = p->trie[ti];
        d.key_off = take(int64_t(p->k) * 4);
        d.uniq_off = take(int64_t(d.kv) * 8);
        d.rep_off = take(int64_t(d.kv) * 4);
        d.uL_off = d.uR_off = d.gstart_off = -1;
        d.l_key_off = d.r_key_off = -1;
        if (v >= L) {
            d.uL_off = take(int64_t(d.kv) * 4);
            d.uR_off = take(int64_t(d.kv) * 4);
            d.kL = int(an.nodes[an.nodes[v].l].kv);
            d.gstart_off = take(int64_t(d.kL + 1) * 4);
        }
    }
    for (int v = L; v < N; ++v) {
        const int ti = p->trie_of_node[v];
        if (ti < 0) continue;
        xebk::TrieDesc& d = p->trie[ti];
        const int tl = p->trie_of_node[an.nodes[v].l], tr = p->trie_of_node[an.nodes[v].r];
        d.l_key_off = tl >= 0 ? p->trie[tl].key_off : -1;
        d.r_key_off = tr >= 0 ? p->trie[tr].key_off : -1;
        p->trie_internal.push_back(ti);
    }
    p->t_acc = take((an.nodes[N - 1].kv << p->w) * 16);
    p->t_amps = take((int64_t(p->k) << p->w) * 16);
    p->t_partials = take(int64_t(p->n_xeb_blocks) * 16);
    p->t_result = take(64);
    p->t_err = take(16);
    p->t_sort = take(p->k > size_t(xebk::kMaxTrieK) ? int64_t(xebk::trie_sort_scratch_bytes(int(p->k))) : 16);
    {   // memo-level contractions: per-group A offsets + packed B vectors (largest op)
        size_t mx = 16;
        for (const Op& op : p->prog.ops)
            if (op.kind != OP_PERM && op.kv >= 1) {
                if (op.N == 1 && op.kv > 1)
                    mx = std::max(mx, xebk::memo_scratch_bytes(std::max(an.nodes[op.a_node].kv, an.nodes[op.b_node].kv),
                                                               op.kv, op.K, p->elem));
                if (xebk::keyed_fits(op.M, op.N, op.K))   // keyed form, single-key contractions included
                    mx = std::max(mx, xebk::keyed_scratch_bytes(an.nodes[op.b_node].kv, op.K, op.N));
            }
        p->t_memo = take(int64_t(mx));
        p->memo_bytes = mx;
    }
    p->tables_bytes = t;
    p->bytes_total = size_t(off + t);
}

}  // namespace

// Norm-keeping rounding of a leaf to single precision (see xeb.h,
// xeb_round_keep_norm): nearest values first, then, cheapest first, values
// move to their other neighbour while that brings sum y^2 closer to sum x^2.
extern "C" void xeb_round_keep_norm(const double* x, size_t n, float* y) {
    if (!x || !y) return;
    long double err = 0;
    std::vector<std::pair<double, size_t>> cand;
    std::vector<float> other(n);
    for (size_t i = 0; i < n; ++i) {
        const float r = float(x[i]);
        y[i] = r;
        err += (long double)r * r - (long double)x[i] * x[i];
        if (double(r) == x[i] || !std::isfinite(r)) continue;
        other[i] = std::nextafter(r, double(r) > x[i] ? -INFINITY : INFINITY);
        cand.push_back({std::fabs(double(other[i]) - x[i]) - std::fabs(double(r) - x[i]), i});
    }
    std::sort(cand.begin(), cand.end());
    for (const auto& c : cand) {
        const size_t i = c.second;
        const long double d = (long double)other[i] * other[i] - (long double)y[i] * y[i];
        if (std::fabs(double(err + d)) < std::fabs(double(err))) {
            err += d;
            y[i] = other[i];
        }
    }
}

namespace {

// Device values of one constant tensor (a leaf or a folded subtree): complex64
// plans round with xeb_round_keep_norm (opts.reserved[1] = 0 or 2) or to
// nearest (1); an FP64 plan keeps the exact values (0) or takes those
// single-precision values (1, 2: the error the rounding alone causes).
void constant_to_device(const xeb_plan_s* p, const std::vector<cd>& t, char* dst) {
    const int mode = p->opts.reserved[1];
    std::vector<double> x(2 * t.size());
    std::vector<float> y(x.size());
    for (size_t e = 0; e < t.size(); ++e) {
        x[2 * e] = t[e].real();
        x[2 * e + 1] = t[e].imag();
    }
    const bool single = p->elem == 8 || mode != 0;
    if (single && mode == 1) {
        for (size_t i = 0; i < x.size(); ++i) y[i] = float(x[i]);
    } else if (single) {
        xeb_round_keep_norm(x.data(), x.size(), y.data());
    }
    if (p->elem == 8) {
        std::memcpy(dst, y.data(), y.size() * sizeof(float));
    } else {
        double* d = reinterpret_cast<double*>(dst);
        for (size_t i = 0; i < x.size(); ++i) d[i] = single ? double(y[i]) : x[i];
    }
}

std::vector<char> leaf_host_data(xeb_plan_s* p) {
    std::vector<char> h(size_t(p->leafdata_elems) * p->elem);
    for (size_t j = 0; j < p->net.leaves.size(); ++j)
        constant_to_device(p, p->net.leaves[j].t, h.data() + size_t(p->leaf_src_off[j]) * p->elem);
    return h;
}

// the folded constants, one after another in fold_roots order
std::vector<char> fold_host_data(xeb_plan_s* p) {
    size_t n = 0;
    for (const auto& v : p->fold_vals) n += v.size();
    std::vector<char> h(n * p->elem);
    size_t at = 0;
    for (const auto& v : p->fold_vals) {
        constant_to_device(p, v, h.data() + at);
        at += v.size() * p->elem;
    }
    return h;
}

// Keyed SIMT form (keyed.cu): complex64, k_v > 1 keys grouped by left key (or
// one group), K in {4, 8, 16, 32}, N in {1, 2, 4, 8, 16}, M a multiple of 32,
// row-major results at even float2 offsets, summed bits below address bit 31.
// single: also contractions with one key (one left-key group; every row of
// A multiplied by the one B)
bool keyed_ok(const xeb_plan_s* p, const Op& op, const xebk::GemmDesc& d, bool single = false) {
    if (p->elem != 8 || op.kv < 1 || (op.kv == 1 && !single) || !xebk::keyed_fits(op.M, op.N, op.K) || !d.c_natural)
        return false;
    if (!d.gstart && d.n_groups != 1) return false;
    if (d.c_off % 2 != 0 || d.c_key % 2 != 0) return false;
    for (int i = 0; i < d.nak; ++i)
        if (d.apk[i] > 30) return false;
    return xebk::keyed_scratch_bytes(p->an.nodes[op.b_node].kv, op.K, op.N) <= p->memo_bytes;
}

// Rows per lane of the keyed form when the autotuner has not chosen: two
// wherever they fit (each uniform load of B then feeds twice the
// multiply-adds).
bool keyed_rows2_default(const Op& op) { return op.K <= 16; }

// Kernel form of one contraction: CH_AUTO follows the options; the others
// force a form (the autotuner's candidates).  False if the form does not fit.
bool select_kernel(xeb_plan_s* p, const Op& op, int ch, GemmLaunch& g) {
    char* tables = p->ws + p->off_tables;
    const xebk::GemmDesc& d = g.d;
    const bool tf32 = p->opts.precision == XEB_PREC_TF32X3;
    auto tc_common = [&](bool grouped) {
        g.tc.a_off = d.a_off;
        g.tc.b_off = grouped ? 0 : d.b_off;
        g.tc.c_off = d.c_off;
        g.tc.err = reinterpret_cast<int32_t*>(tables + p->t_err);
        g.tc.split_bits = p->opts.split_bits > 0 ? p->opts.split_bits : kSplitBitsDefault;
        g.tc.split_terms = p->opts.split_terms > 0 ? p->opts.split_terms : kSplitTermsDefault;
        g.tc.wait_ns = uint64_t(p->opts.timeout_ms > 0 ? p->opts.timeout_ms : kTimeoutMsDefault) * 1000000ull;
        g.tc.test_wait = p->test_wait;
        std::memset(&g.tmap, 0, sizeof(g.tmap));
    };
    if (op.M == 1 && op.N == 1) {
        g.kernel = xebk::GK_TAIL;
        return ch == CH_AUTO || ch == CH_SIMT;
    }
    const bool tc_ok = tf32 && (ch == CH_AUTO || ch == CH_TC2 || ch == CH_TC2_GATHER);
    if (tc_ok && tc_tile(op, g.tc, xebk::kTc2RowBits, true)) {
        g.kernel = GK_TC2;
        tc_common(false);
        const bool gather = ch == CH_TC2_GATHER || (ch == CH_AUTO && p->opts.reserved[3] == 1);
        if (g.tc.tma && (gather || !encode_a_map(g.tc, reinterpret_cast<const float2*>(p->ws + p->off_arena), g.tmap)))
            g.tc.tma = 0;
        return !(ch == CH_TC2 && !g.tc.tma);   // CH_TC2 means the TMA form
    }
    // keyed tensor-core form: an autotuner choice, or the default with
    // opts.reserved[6] = 1 (on the 53-qubit plans, whose keyed contractions
    // are mostly K = N = 16, it ran no faster than the SIMT kernels)
    if (tc_ok && (ch == CH_TC2_GATHER || (ch == CH_AUTO && p->opts.reserved[6] == 1)) &&
        tc_keyed(op, d, g.tc)) {
        g.kernel = GK_TC2;
        tc_common(false);
        return true;
    }
    if (tf32 && (ch == CH_AUTO || ch == CH_TCKD) && tc_kdeep(op, d, g.kd)) {
        g.kernel = GK_TCKD;
        g.kd.err = reinterpret_cast<int32_t*>(tables + p->t_err);
        g.kd.split_bits = p->opts.split_bits > 0 ? p->opts.split_bits : kSplitBitsDefault;
        g.kd.split_terms = p->opts.split_terms > 0 ? p->opts.split_terms : kSplitTermsDefault;
        g.kd.wait_ns = uint64_t(p->opts.timeout_ms > 0 ? p->opts.timeout_ms : kTimeoutMsDefault) * 1000000ull;
        g.kd.test_wait = p->test_wait;
        return true;
    }
    if (ch == CH_TCKD) return false;
    if (tc_ok && ch != CH_AUTO) return false;
    if (tf32 && (ch == CH_GROUPED || (ch == CH_AUTO && p->opts.reserved[4] == 1)) &&
        tc_grouped(p->an, op, d, g.tc)) {
        g.kernel = GK_TC2;
        tc_common(true);
        g.tc.grp_a = reinterpret_cast<const int64_t*>(tables + p->t_memo);
        g.tc.bpack_off = (p->off_tables + p->t_memo + ((d.n_groups * 8 + 255) & ~int64_t(255))) / 8;
        g.s = xebk::StreamDesc{};
        return true;
    }
    // keyed contractions with few summed values and narrow results, complex64
    // (keyed.cu): the default SIMT form where it fits
    // single-key contractions take the keyed form by default where it measured
    // faster than the streaming kernel (30-qubit plans: K = N = 4, 8, 16; the
    // streaming kernel stays faster for K = 4, N = 16)
    const bool keyed_default = op.kv > 1 || op.K >= 8 || op.N <= 4;
    if (((ch == CH_AUTO && keyed_default) || ch == CH_KEYED || ch == CH_KEYED2) && keyed_ok(p, op, d, true)) {
        const bool rows2 = xebk::keyed_fits_rows2(op.M, op.N, op.K);
        if (ch == CH_KEYED2 && !rows2) return false;
        g.kernel = xebk::GK_KEYED;
        g.kvB = p->an.nodes[op.b_node].kv;
        g.rpt = ch == CH_KEYED2 || (ch == CH_AUTO && rows2 && keyed_rows2_default(op)) ? 2 : 1;
        return true;
    }
    if (ch == CH_KEYED || ch == CH_KEYED2) return false;
    const bool shape_ch = ch == CH_STREAM_N2 || ch == CH_STREAM_HALF;
    if (ch != CH_AUTO && ch != CH_SIMT && !shape_ch) return false;
    // few summed values and wide results: the stores dominate, so by default
    // two result columns per thread (a warp writes whole result rows)
    const bool wide_store = op.K <= 4 && op.N >= 32;
    if (stream_tile(op, p->elem, g.s, ch == CH_STREAM_N2 || (ch == CH_AUTO && wide_store) ? 2 : 0,
                    ch == CH_STREAM_HALF)) {
        g.kernel = op.N == 1 && op.kv > 1 && d.gstart ? xebk::GK_MEMO : xebk::GK_STREAM;
        if (shape_ch && g.kernel != xebk::GK_STREAM) return false;
    } else if (shape_ch) return false;
    // N = 1 with a deep sum over few rows: a warp per output (the GEMV kernel
    // would run one long dependent chain per thread on a nearly idle GPU)
    else if (op.N == 1 && op.K >= 128 && op.M <= 64) g.kernel = xebk::GK_TAIL;
    else if (op.N == 1) g.kernel = xebk::GK_GEMV;
    else if (op.K >= 32 && std::min(op.M, op.N) <= xebk::kKdTile && d.c_natural) g.kernel = xebk::GK_KDEEP;
    else if (op.M >= 16 && op.N >= 16) g.kernel = xebk::GK_TILED;
    else g.kernel = xebk::GK_GENERIC;
    return true;
}

void build_launches(xeb_plan_s* p) {
    const Analysis& an = p->an;
    const Program& pr = p->prog;
    const int L = an.L;
    char* tables = p->ws + p->off_tables;
    // leaves (those inside folded subtrees are never materialised)
    p->leafdesc.clear();
    p->leafdesc_leaf.clear();
    for (int j = 0; j < L; ++j) {
        if (!p->folded.empty() && p->folded[size_t(j)]) continue;
        const Leaf& lf = p->net.leaves[j];
        p->leafdesc_leaf.push_back(j);
        p->leafdesc.push_back(xebk::LeafDesc{});
        xebk::LeafDesc& d = p->leafdesc.back();
        d.dst_off = pr.bufs[pr.node_buf[j]].off;
        d.src_off = p->leaf_src_off[j];
        const std::vector<int>& lay = pr.layout[j];
        d.r = int(lay.size());
        d.n_out = int(lf.out_q.size());
        d.n_canon = d.n_out + int(lf.legs.size());
        d.kv = int(an.nodes[j].kv);
        for (int b = 0; b < d.r; ++b) {
            const int leg = lay[d.r - 1 - b];
            const int axis = d.n_out + int(std::find(lf.legs.begin(), lf.legs.end(), leg) - lf.legs.begin());
            d.src_pos[b] = d.n_canon - 1 - axis;
        }
        d.n_sl = 0;
        for (size_t a = 0; a < lf.legs.size(); ++a) {
            const auto it = std::find(p->sliced.begin(), p->sliced.end(), lf.legs[a]);
            if (it == p->sliced.end()) continue;
            d.sl_pos[d.n_sl] = d.n_canon - 1 - (d.n_out + int(a));
            d.sl_bit[d.n_sl] = int(it - p->sliced.begin());
            ++d.n_sl;
        }
        const int ti = p->trie_of_node[j];
        d.uniq_off = ti >= 0 ? p->trie[ti].uniq_off : -1;
    }
    // ops
    p->perms.assign(pr.ops.size(), xebk::PermDesc{});
    p->gemms.assign(pr.ops.size(), GemmLaunch{});
    for (size_t i = 0; i < pr.ops.size(); ++i) {
        const Op& op = pr.ops[i];
        if (op.kind == OP_PERM) {
            xebk::PermDesc& d = p->perms[i];
            d.r = op.r;
            d.keys = op.keys;
            const int r = op.r;
            std::vector<int> pinv(r);
            for (int j = 0; j < r; ++j) pinv[op.perm[j]] = j;
            const int t0 = std::min(r, 5);
            std::vector<int> U;
            for (int j = 0; j < t0; ++j) U.push_back(j);
            for (int j = 0; j < t0; ++j)
                if (std::find(U.begin(), U.end(), op.perm[j]) == U.end()) U.push_back(op.perm[j]);
            for (int j = 0; j < r && int(U.size()) < std::min(r, 8); ++j)
                if (std::find(U.begin(), U.end(), j) == U.end()) U.push_back(j);
            d.u = int(U.size());
            for (int i2 = 0; i2 < d.u; ++i2) d.usrc[i2] = U[i2];
            std::vector<int> Ud;
            for (int j = 0; j < t0; ++j) Ud.push_back(j);
            for (int i2 = 0; i2 < d.u; ++i2) {
                const int dp = pinv[U[i2]];
                if (std::find(Ud.begin(), Ud.end(), dp) == Ud.end()) Ud.push_back(dp);
            }
            for (int i2 = 0; i2 < d.u; ++i2) {
                d.udst[i2] = Ud[i2];
                const int sp = op.perm[Ud[i2]];
                d.udst_e[i2] = int(std::find(U.begin(), U.end(), sp) - U.begin());
            }
            d.n_outer = 0;
            for (int j = 0; j < r; ++j)
                if (std::find(U.begin(), U.end(), j) == U.end()) {
                    d.outer_src[d.n_outer] = j;
                    d.outer_dst[d.n_outer] = pinv[j];
                    ++d.n_outer;
                }
        } else {
            GemmLaunch& g = p->gemms[i];
            xebk::GemmDesc& d = g.d;
            d.M = op.M;
            d.N = op.N;
            d.K = op.K;
            d.kv = op.kv;
            d.a_off = pr.bufs[op.a_buf].off;
            d.b_off = pr.bufs[op.b_buf].off;
            d.c_off = pr.bufs[op.c_buf].off;
            d.a_key = int64_t(1) << op.a_rank;
            d.b_key = int64_t(1) << op.b_rank;
            d.c_key = op.M * op.N;
            d.nam = int(op.a_pos_m.size());
            d.nak = int(op.a_pos_k.size());
            d.nbk = int(op.b_pos_k.size());
            d.nbn = int(op.b_pos_n.size());
            for (int t = 0; t < d.nam; ++t) d.apm[t] = int8_t(op.a_pos_m[t]);
            for (int t = 0; t < d.nak; ++t) d.apk[t] = int8_t(op.a_pos_k[t]);
            for (int t = 0; t < d.nbk; ++t) d.bpk[t] = int8_t(op.b_pos_k[t]);
            for (int t = 0; t < d.nbn; ++t) d.bpn[t] = int8_t(op.b_pos_n[t]);
            d.c_natural = 1;
            for (int t = 0; t < d.nam; ++t) {
                d.cpm[t] = int8_t(op.c_pos_m[t]);
                if (op.c_pos_m[t] != d.nbn + t) d.c_natural = 0;
            }
            for (int t = 0; t < d.nbn; ++t) {
                d.cpn[t] = int8_t(op.c_pos_n[t]);
                if (op.c_pos_n[t] != t) d.c_natural = 0;
            }
            const int ti = p->trie_of_node[op.node];
            if (ti >= 0) {
                const xebk::TrieDesc& t = p->trie[ti];
                d.uL = reinterpret_cast<const int32_t*>(tables + t.uL_off);
                d.uR = reinterpret_cast<const int32_t*>(tables + t.uR_off);
                d.gstart = reinterpret_cast<const int32_t*>(tables + t.gstart_off);
                d.n_groups = t.kL;
            } else {
                d.uL = d.uR = d.gstart = nullptr;
                d.n_groups = 1;
            }
            select_kernel(p, op, p->choice.empty() ? CH_AUTO : p->choice[i], g);
        }
    }
}

// Every element a launch can touch must lie inside the buffers it names.
bool validate_launches(const xeb_plan_s* p, std::string& why) {
    const Program& pr = p->prog;
    const Analysis& an = p->an;
    auto inside = [&](int buf, int64_t lo, int64_t hi) {
        const Buffer& b = pr.bufs[buf];
        return lo >= b.off && hi < b.off + b.elems && b.off + b.elems <= pr.arena_elems;
    };
    for (size_t i = 0; i < pr.ops.size(); ++i) {
        const Op& op = pr.ops[i];
        if (op.kind == OP_PERM) {
            const xebk::PermDesc& d = p->perms[i];
            std::vector<int> seen_s(d.r, 0), seen_d(d.r, 0);
            for (int t = 0; t < d.u; ++t) { ++seen_s[d.usrc[t]]; ++seen_d[d.udst[t]]; }
            for (int t = 0; t < d.n_outer; ++t) { ++seen_s[d.outer_src[t]]; ++seen_d[d.outer_dst[t]]; }
            for (int t = 0; t < d.r; ++t)
                if (seen_s[t] != 1 || seen_d[t] != 1) { why = "permutation bits"; return false; }
            const int64_t n = d.keys << d.r;
            if (!inside(op.src_buf, pr.bufs[op.src_buf].off, pr.bufs[op.src_buf].off + n - 1) ||
                !inside(op.dst_buf, pr.bufs[op.dst_buf].off, pr.bufs[op.dst_buf].off + n - 1)) {
                why = "permutation buffer";
                return false;
            }
            continue;
        }
        const xebk::GemmDesc& g = p->gemms[i].d;
        const int64_t ka = an.nodes[op.a_node].kv, kb = an.nodes[op.b_node].kv;
        auto perm_ok = [](const int8_t* a, int na, const int8_t* b, int nb, int rank) {
            if (na + nb != rank) return false;
            std::vector<int> seen(rank, 0);
            for (int t = 0; t < na; ++t) { if (a[t] < 0 || a[t] >= rank) return false; ++seen[a[t]]; }
            for (int t = 0; t < nb; ++t) { if (b[t] < 0 || b[t] >= rank) return false; ++seen[b[t]]; }
            for (int t = 0; t < rank; ++t) if (seen[t] != 1) return false;
            return true;
        };
        if (!perm_ok(g.apm, g.nam, g.apk, g.nak, op.a_rank) || !perm_ok(g.bpk, g.nbk, g.bpn, g.nbn, op.b_rank) ||
            g.nak != g.nbk || (int64_t(1) << g.nam) != g.M || (int64_t(1) << g.nbn) != g.N ||
            (int64_t(1) << g.nak) != g.K) {
            why = "gemm index positions of node " + std::to_string(op.node);
            return false;
        }
        const int64_t a_hi = g.a_off + ka * g.a_key - 1;
        const int64_t b_hi = g.b_off + kb * g.b_key - 1;
        const int64_t c_hi = g.c_off + g.kv * g.c_key - 1;
        if (!inside(op.a_buf, g.a_off, a_hi) || !inside(op.b_buf, g.b_off, b_hi) || !inside(op.c_buf, g.c_off, c_hi)) {
            why = "gemm operand of node " + std::to_string(op.node);
            return false;
        }
        if ((ka > 1 || kb > 1) && !g.uL) { why = "gemm without key tables"; return false; }
        {
            const int rc = g.nam + g.nbn;
            std::vector<int> seen(rc, 0);
            for (int t2 = 0; t2 < g.nam; ++t2)
                if (g.cpm[t2] < 0 || g.cpm[t2] >= rc || seen[g.cpm[t2]]++) { why = "result positions"; return false; }
            for (int t2 = 0; t2 < g.nbn; ++t2)
                if (g.cpn[t2] < 0 || g.cpn[t2] >= rc || seen[g.cpn[t2]]++) { why = "result positions"; return false; }
            if (!g.c_natural && p->gemms[i].kernel != GK_TC2 && p->gemms[i].kernel != GK_TCKD) {
                why = "non row-major result for a kernel that writes row-major only (node " +
                      std::to_string(op.node) + ")";
                return false;
            }
        }
        if (p->gemms[i].kernel == GK_TCKD) {
            const xebk::KdDesc& k = p->gemms[i].kd;
            bool bad = k.M != g.M || k.N != g.N || (k.M != 16 && k.M != 32) || (k.N != 16 && k.N != 32) ||
                       k.K != g.K || k.K < 64 || k.K % 64 != 0 || k.K > 8192 || k.kv != g.kv || !k.uL || !k.uR ||
                       k.a_off != g.a_off ||
                       k.b_off != g.b_off || k.c_off != g.c_off || k.a_key != g.a_key || k.b_key != g.b_key ||
                       k.c_key != g.c_key || k.nak != g.nak || k.nbk != g.nbk || !k.err || k.wait_ns == 0 ||
                       k.split_bits < 8 || k.split_bits > 11 || (k.split_terms != 3 && k.split_terms != 4);
            for (int t2 = 0; t2 < g.nam && !bad; ++t2) bad = k.apm[t2] != g.apm[t2] || k.cpm[t2] != g.cpm[t2];
            for (int t2 = 0; t2 < g.nbn && !bad; ++t2) bad = k.bpn[t2] != g.bpn[t2] || k.cpn[t2] != g.cpn[t2];
            for (int t2 = 0; t2 < g.nak && !bad; ++t2) bad = k.apk[t2] != g.apk[t2] || k.bpk[t2] != g.bpk[t2];
            if (bad) {
                why = "deep-K tensor-core form of node " + std::to_string(op.node);
                return false;
            }
        }
        if (p->gemms[i].kernel == GK_TC2) {
            const xebk::TcDesc& t = p->gemms[i].tc;
            const int row_bits = xebk::kTc2RowBits;
            // grouped memo-level form: the columns are a group's keys (N2/2 of them at most)
            const bool grp = t.grp;
            const bool keyed = grp && t.keyed;   // keyed form: the op's own K x N per key
            const bool mgrp = grp && !t.keyed;   // memo-level groups: keys as columns
            int lnp = 0;
            while ((2 << lnp) < t.N2) ++lnp;
            const int64_t gN = mgrp ? t.N2 / 2 : g.N;
            const int nbn_eff = mgrp ? lnp : g.nbn;
            if (t.M != g.M || t.M % (int64_t(1) << row_bits) != 0 || t.K2 != 2 * g.K || t.N2 != 2 * gN ||
                t.K2 % 32 != 0 || t.N2 % 32 != 0 || t.N2 > 128 || t.K2 > 128 || t.n_chunks * 32 != t.K2 ||
                t.n_chunks > 4 || t.T != row_bits + 4 || (!grp && g.kv != 1) || t.split_bits < 8 ||
                t.split_bits > 11 || (t.split_terms != 3 && t.split_terms != 4) || t.wait_ns == 0) {
                why = "tensor-core tile of node " + std::to_string(op.node);
                return false;
            }
            if (keyed && (t.tma || (t.tpg << row_bits) != g.M || t.n_groups != g.kv || t.c_key != g.c_key ||
                          t.a_key != g.a_key || t.b_key != g.b_key || t.uL != g.uL || t.uR != g.uR)) {
                why = "keyed tensor-core form of node " + std::to_string(op.node);
                return false;
            }
            if (mgrp && (t.tma || (t.tpg << row_bits) != g.M || t.n_groups != g.n_groups || t.c_key != g.M ||
                        t.N2 / 2 < an.nodes[op.b_node].kv || t.n_groups != an.nodes[op.a_node].kv ||
                        xebk::memo_scratch_bytes(t.n_groups, g.kv, g.K, 8) > p->memo_bytes ||
                        !inside(op.c_buf, t.c_off, t.c_off + g.kv * t.c_key - 1))) {
                why = "grouped tensor-core form of node " + std::to_string(op.node);
                return false;
            }
            if (!grp && !inside(op.c_buf, t.c_off, t.c_off + g.M * g.N - 1)) {
                why = "tensor-core operand of node " + std::to_string(op.node);
                return false;
            }
            for (int i = 0; i < t.T; ++i)
                if (t.pos[i] < 0 || t.pos[i] >= op.a_rank) { why = "tensor-core tile positions"; return false; }
            {
                const int rc = g.nam + nbn_eff;
                if (t.n_ext + row_bits != g.nam || t.n_ext > 32 || t.Tst != row_bits + nbn_eff || t.Tst < row_bits + 4 ||
                    t.Tst > 16) {
                    why = "tensor-core result tile of node " + std::to_string(op.node);
                    return false;
                }
                std::vector<int> seen(rc, 0);
                for (int i2 = 0; i2 < t.n_ext; ++i2)
                    if (t.ext_cpos[i2] < 0 || t.ext_cpos[i2] >= rc || seen[t.ext_cpos[i2]]++) { why = "tc ext"; return false; }
                for (int i2 = 0; i2 < t.Tst; ++i2)
                    if (t.st_pos[i2] < 0 || t.st_pos[i2] >= rc || seen[t.st_pos[i2]]++) { why = "tc store"; return false; }
                int64_t ahi = 0;
                for (int i2 = 0; i2 < t.n_ext; ++i2) ahi |= int64_t(1) << t.ext_apos[i2];
                int64_t thi = 0;
                for (int i2 = 0; i2 < t.T; ++i2) thi |= int64_t(1) << t.pos[i2];
                const int64_t akey = grp ? (an.nodes[op.a_node].kv - 1) * g.a_key : 0;   // largest group A offset
                if (!inside(op.a_buf, t.a_off, t.a_off + akey + ahi + thi + t.chunk_off[t.n_chunks - 1])) {
                    why = "tensor-core operand rows of node " + std::to_string(op.node);
                    return false;
                }
                if (t.tma) {  // TMA boxes: rows y .. y + 2^box_log2 - 1 of an [M][K] matrix inside A's buffer
                    bool bad = t.box_log2 < 3 || t.box_log2 > row_bits || t.row_shift != int(op.a_pos_k.size()) ||
                               !inside(op.a_buf, t.a_off, t.a_off + g.M * g.K - 1);
                    int64_t yext = 0;
                    for (int i2 = 0; i2 < t.n_ext && !bad; ++i2) {
                        bad = t.ext_apos[i2] < t.row_shift;
                        if (!bad) yext |= int64_t(1) << (t.ext_apos[i2] - t.row_shift);
                    }
                    for (int j = 0; j < (1 << (row_bits - t.box_log2)) && !bad; ++j)
                        bad = t.box_y[j] < 0 || yext + t.box_y[j] + (int64_t(1) << t.box_log2) > g.M;
                    if (bad) {
                        why = "tensor-core TMA boxes of node " + std::to_string(op.node);
                        return false;
                    }
                }
            }
        }
        if (p->gemms[i].kernel == xebk::GK_KEYED) {
            const GemmLaunch& gl = p->gemms[i];
            if (!keyed_ok(p, op, g, true) || gl.kvB != kb || (kb > 1 && !g.uR) ||
                !(gl.rpt == 1 || (gl.rpt == 2 && xebk::keyed_fits_rows2(g.M, g.N, g.K)))) {
                why = "keyed form of node " + std::to_string(op.node);
                return false;
            }
        }
        if (p->gemms[i].kernel == xebk::GK_MEMO &&
            xebk::memo_scratch_bytes(p->gemms[i].d.n_groups, g.kv, g.K, p->elem) > p->memo_bytes) {
            why = "memo-level scratch of node " + std::to_string(op.node);
            return false;
        }
        if (p->gemms[i].kernel == xebk::GK_STREAM || p->gemms[i].kernel == xebk::GK_MEMO) {
            const xebk::StreamDesc& sd = p->gemms[i].s;
            if (sd.T > 32 || sd.T != sd.tm + g.nak || (1 << sd.tm) != sd.R || sd.R > g.M || sd.R < 1) {
                why = "stream tile of node " + std::to_string(op.node);
                return false;
            }
            for (int t = 0; t < sd.T; ++t)
                if (sd.pos[t] < 0 || sd.pos[t] >= op.a_rank) { why = "stream tile positions"; return false; }
            if (sd.tm > g.nam) { why = "stream tile rows"; return false; }
        }
    }
    for (size_t j = 0; j < p->leafdesc.size(); ++j) {
        const xebk::LeafDesc& d = p->leafdesc[j];
        if (!inside(pr.node_buf[size_t(p->leafdesc_leaf[j])], d.dst_off, d.dst_off + (int64_t(d.kv) << d.r) - 1)) { why = "leaf dst"; return false; }
        if (d.src_off + (int64_t(1) << d.n_canon) > p->leafdata_elems) { why = "leaf src"; return false; }
        for (int b = 0; b < d.r; ++b)
            if (d.src_pos[b] < 0 || d.src_pos[b] >= d.n_canon - d.n_out) { why = "leaf layout"; return false; }
    }
    return true;
}

// one contraction's kernel(s), as chosen by select_kernel
template <typename T>
cudaError_t launch_gemm_op(xeb_plan_s* p, const GemmLaunch& g, T* arena, char* tables, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    if (g.kernel == GK_TCKD) {
        if constexpr (sizeof(T) == 8) e = xebk::launch_tc_kdeep(g.kd, reinterpret_cast<float2*>(arena), p->n_sms, st);
    } else if (g.kernel == GK_TC2) {
        if constexpr (sizeof(T) == 8) {
            if (g.tc.grp) e = xebk::launch_memo_prep<float2>(g.d, reinterpret_cast<float2*>(arena), tables + p->t_memo, st);
            if (e == cudaSuccess) e = xebk::launch_tc_gemm2(g.tc, g.tmap, reinterpret_cast<float2*>(arena), p->n_sms, st);
        }
    } else if (g.kernel == xebk::GK_KEYED) {
        if constexpr (sizeof(T) == 8)
            e = xebk::launch_gemm_keyed(g.d, g.kvB, g.rpt, reinterpret_cast<float2*>(arena), tables + p->t_memo, p->n_sms, st);
        else
            e = cudaErrorInvalidValue;
    } else if (g.kernel == xebk::GK_MEMO) {
        e = xebk::launch_gemm_memo<T>(g.d, g.s, arena, tables + p->t_memo, st);
    } else if (g.kernel == xebk::GK_STREAM) {
        e = xebk::launch_gemm_stream<T>(g.d, g.s, arena, st);
    } else {
        e = xebk::launch_gemm<T>(g.kernel, g.d, arena, st);
    }
    return e;
}

template <typename T>
xeb_status run_slices(xeb_plan_s* p, double2* amps_out, cudaStream_t st) {
    const Analysis& an = p->an;
    const Program& pr = p->prog;
    char* tables = p->ws + p->off_tables;
    T* arena = reinterpret_cast<T*>(p->ws + p->off_arena);
    const T* leafdata = reinterpret_cast<const T*>(p->ws + p->off_leafdata);
    double2* acc = reinterpret_cast<double2*>(tables + p->t_acc);
    const int64_t kv_root = an.nodes.back().kv;
    XEB_CUDA(cudaMemsetAsync(acc, 0, size_t(kv_root << p->w) * 16, st));
    const int64_t n_run = p->slice_all ? int64_t(1) << p->sliced.size() : int64_t(p->slice_ids.size());
    const auto* ldesc = reinterpret_cast<const xebk::LeafDesc*>(tables + p->t_leaf_desc);
    const double es = double(sizeof(T));
    int64_t s_prev = 0;
    for (int64_t si = 0; si < n_run; ++si) {
        const int64_t s = p->slice_all ? si : p->slice_ids[size_t(si)];
        const uint32_t changed = uint32_t(s ^ s_prev);   // slice bits that moved (unused for si = 0)
        s_prev = s;
        {
            ProfScope ps(p, st, XEB_KC_LEAVES, 0.0, 0.0);
            XEB_CUDA(xebk::launch_leaves<T>(ldesc, int(p->leafdesc.size()), leafdata, arena, tables, s, st));
        }
        for (size_t i = 0; i < pr.ops.size(); ++i) {
            const Op& op = pr.ops[i];
            if (op.kind == OP_PERM) {
                ProfScope ps(p, st, XEB_KC_PERMUTE, 0.0, 2.0 * es * double(op.keys) * std::ldexp(1.0, op.r));
                XEB_CUDA(xebk::launch_permute<T>(p->perms[i], arena + pr.bufs[op.src_buf].off,
                                                 arena + pr.bufs[op.dst_buf].off, st));
            } else {
                if (p->op_folded[i]) continue;   // evaluated on the host at plan creation
                if (si > 0 && !(changed & p->node_mask[size_t(op.node)])) continue;   // still holds this slice's value
                const GemmLaunch& g = p->gemms[i];
                const double ka = double(an.nodes[op.a_node].kv), kb = double(an.nodes[op.b_node].kv);
                const double fl = 8.0 * double(op.kv) * double(op.M) * double(op.N) * double(op.K);
                const double by = es * (ka * double(op.M) * double(op.K) + kb * double(op.K) * double(op.N) +
                                        double(op.kv) * double(op.M) * double(op.N));
                static const int cls_of[8] = {XEB_KC_GEMM_GENERIC, XEB_KC_GEMM_TILED, XEB_KC_GEMM_GEMV,
                                              XEB_KC_GEMM_TAIL,    XEB_KC_GEMM_STREAM, XEB_KC_GEMM_MEMO,
                                              XEB_KC_GEMM_KDEEP,   XEB_KC_GEMM_KEYED};
                ProfScope ps(p, st, g.kernel == GK_TCKD ? XEB_KC_GEMM_TC_KDEEP : g.kernel >= GK_TC2 ? XEB_KC_GEMM_TC : cls_of[g.kernel],
                             fl, by, int(i));
                XEB_CUDA(launch_gemm_op<T>(p, g, arena, tables, st));
            }
        }
        {
            ProfScope ps(p, st, XEB_KC_ACCUM, 0.0, double(kv_root << p->w) * (16.0 + 2 * es));
            XEB_CUDA(xebk::launch_root_accum<T>(arena + pr.bufs[pr.node_buf.back()].off, acc, kv_root << p->w, st));
        }
    }
    const int troot = p->trie_of_node[int(an.nodes.size()) - 1];
    const int32_t* key_root = reinterpret_cast<const int32_t*>(tables + p->trie[troot].key_off);
    ProfScope ps(p, st, XEB_KC_XEB, 0.0, double(p->k) * 4.0 + double(p->k << p->w) * 32.0);
    XEB_CUDA(xebk::launch_gather_xeb(acc, key_root, int64_t(p->k), p->rootmap, amps_out,
                                     reinterpret_cast<double*>(tables + p->t_partials), p->n_xeb_blocks,
                                     reinterpret_cast<double*>(tables + p->t_result), p->net.n, st));
    return XEB_OK;
}

xeb_status build_tables(xeb_plan_s* p, cudaStream_t st) {
    char* tables = p->ws + p->off_tables;
    ProfScope ps(p, st, XEB_KC_TRIE, 0.0, double(p->k) * 8.0 * double(p->trie.size() + 1));
    const auto* tdesc = reinterpret_cast<const xebk::TrieDesc*>(tables + p->t_trie_desc);
    if (p->k <= size_t(xebk::kMaxTrieK))
        XEB_CUDA(xebk::launch_trie_keys(tdesc, int(p->trie.size()),
                                        reinterpret_cast<const uint64_t*>(tables + p->t_bits), int(p->k),
                                        reinterpret_cast<const int32_t*>(tables + p->t_pi), tables,
                                        reinterpret_cast<int32_t*>(tables + p->t_err), st));
    else
        XEB_CUDA(xebk::launch_trie_keys_large(tdesc, p->trie.data(), int(p->trie.size()),
                                              reinterpret_cast<const uint64_t*>(tables + p->t_bits), int(p->k),
                                              reinterpret_cast<const int32_t*>(tables + p->t_pi), tables,
                                              tables + p->t_sort, reinterpret_cast<int32_t*>(tables + p->t_err), st));
    XEB_CUDA(xebk::launch_trie_links(tdesc, reinterpret_cast<const int*>(tables + p->t_internal),
                                     int(p->trie_internal.size()), p->max_kv, tables, st));
    p->tables_ready = true;
    return XEB_OK;
}

xeb_status check_bound(xeb_plan_s* p) {
    if (!p) return fail(XEB_EINVAL, "NULL plan");
    if (!p->bound) return fail(XEB_EINVAL, "plan not bound to device memory (call xeb_plan_bind)");
    return XEB_OK;
}

}  // namespace

extern "C" size_t xeb_plan_device_bytes(xeb_plan_s* p) {
    if (!p) return 0;
    if (p->bytes_total == 0) layout_device(p);
    return p->bytes_total;
}

extern "C" xeb_status xeb_plan_bind(xeb_plan_s* p, void* workspace, size_t bytes, uintptr_t stream) {
    if (!p) return fail(XEB_EINVAL, "NULL plan");
    if (p->bound) return fail(XEB_EINVAL, "plan already bound");
    for (const Buffer& b : p->prog.bufs)
        if (b.elems >= xebp::kSatElems)
            return fail(XEB_ENOMEM, "plan has a tensor of 2^48 or more elements: it fits no device (slice more legs)");
    layout_device(p);
    {
        int dev = 0, sms = 0;
        XEB_CUDA(cudaGetDevice(&dev));
        XEB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        p->n_sms = sms > 0 ? sms : 152;
        if (p->opts.precision == XEB_PREC_TF32X3) {
            int major = 0, minor = 0;
            XEB_CUDA(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev));
            XEB_CUDA(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev));
            if (major != 10 || minor != 3)
                return fail(XEB_EUNSUPPORTED, "TF32x3 tensor-core path is built for sm_103a only");
        }
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (workspace) {
        if (bytes < p->bytes_total) return fail(XEB_ENOMEM, "workspace smaller than xeb_plan_device_bytes()");
        if (reinterpret_cast<uintptr_t>(workspace) % 256) return fail(XEB_EINVAL, "workspace must be 256-byte aligned");
        p->ws = static_cast<char*>(workspace);
        p->owns = false;
    } else {
        void* w = nullptr;
        cudaError_t e = cudaMalloc(&w, p->bytes_total);
        if (e != cudaSuccess) return fail(XEB_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        p->ws = static_cast<char*>(w);
        p->owns = true;
    }
    p->ws_bytes = p->bytes_total;
    XEB_CUDA(xebk::prepare_kernels());
    build_launches(p);
    {
        std::string why;
        if (!validate_launches(p, why)) {
            if (p->owns) cudaFree(p->ws);
            p->ws = nullptr;
            return fail(XEB_EINVAL, "internal layout check failed: " + why);
        }
    }
    char* tables = p->ws + p->off_tables;
    // constant tables (host copies kept alive in the plan until the copies finish)
    const std::vector<char> leafdata = leaf_host_data(p);
    std::vector<int32_t> pi(p->an.pi.begin(), p->an.pi.end());
    XEB_CUDA(cudaMemcpyAsync(p->ws + p->off_leafdata, leafdata.data(), leafdata.size(), cudaMemcpyHostToDevice, st));
    // folded constants: into their (reserved) arena buffers, once
    const std::vector<char> foldbytes = fold_host_data(p);
    for (size_t f = 0, at = 0; f < p->fold_roots.size(); ++f) {
        const size_t n = p->fold_vals[f].size() * p->elem;
        const int64_t off = p->prog.bufs[size_t(p->prog.node_buf[size_t(p->fold_roots[f])])].off;
        XEB_CUDA(cudaMemcpyAsync(p->ws + p->off_arena + off * int64_t(p->elem), foldbytes.data() + at, n,
                                 cudaMemcpyHostToDevice, st));
        at += n;
    }
    XEB_CUDA(cudaMemcpyAsync(tables + p->t_trie_desc, p->trie.data(), p->trie.size() * sizeof(xebk::TrieDesc),
                             cudaMemcpyHostToDevice, st));
    XEB_CUDA(cudaMemcpyAsync(tables + p->t_internal, p->trie_internal.data(), p->trie_internal.size() * 4,
                             cudaMemcpyHostToDevice, st));
    XEB_CUDA(cudaMemcpyAsync(tables + p->t_leaf_desc, p->leafdesc.data(), p->leafdesc.size() * sizeof(xebk::LeafDesc),
                             cudaMemcpyHostToDevice, st));
    XEB_CUDA(cudaMemcpyAsync(tables + p->t_pi, pi.data(), pi.size() * 4, cudaMemcpyHostToDevice, st));
    XEB_CUDA(cudaMemcpyAsync(tables + p->t_bits, p->bits.data(), p->k * 8, cudaMemcpyHostToDevice, st));
    XEB_CUDA(cudaMemsetAsync(tables + p->t_err, 0, 4, st));
    XEB_CUDA(cudaStreamSynchronize(st));
    p->bound = true;
    return XEB_OK;
}

extern "C" xeb_status xeb_set_bitstrings(xeb_plan_s* p, const uint64_t* bits_dev, size_t k, uintptr_t stream) {
    xeb_status s = check_bound(p);
    if (s != XEB_OK) return s;
    if (k != p->k) return fail(XEB_EINVAL, "k differs from the plan's k");
    if (!bits_dev) return fail(XEB_EINVAL, "bitstrings pointer is NULL");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    char* tables = p->ws + p->off_tables;
    XEB_CUDA(cudaMemcpyAsync(tables + p->t_bits, bits_dev, k * 8, cudaMemcpyDeviceToDevice, st));
    p->tables_ready = false;  // rebuilt by the next step (a1 runs inside it)
    return XEB_OK;
}

namespace {
// One whole step: memo key tables (a1) then every slice (a2-a6) and the XEB
// fold (a7).
xeb_status enqueue_step(xeb_plan_s* p, double2* out, cudaStream_t st) {
    xeb_status s = build_tables(p, st);
    if (s != XEB_OK) return s;
    return p->elem == 8 ? run_slices<float2>(p, out, st) : run_slices<double2>(p, out, st);
}
}  // namespace

namespace {
// Capture one step into g (its profiled form when p->profiling is on).
xeb_status capture_step(xeb_plan_s* p, xeb_plan_s::StepGraph& g, double2* out) {
    drop_graph(p, g);
    if (!p->cap_stream) XEB_CUDA(cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking));
    if (p->profiling) {  // two events per launch, created before the capture opens
        const size_t launches = 2 + (size_t(1) << p->sliced.size()) * (p->prog.ops.size() + 2);
        while (p->event_pool.size() < 2 * launches) {
            cudaEvent_t e = nullptr;
            XEB_CUDA(cudaEventCreate(&e));
            p->event_pool.push_back(e);
        }
    }
    XEB_CUDA(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal));
    std::vector<xeb_plan_s::Rec> outside;
    outside.swap(p->pending);
    p->capturing_prof = p->profiling;
    xeb_status s = enqueue_step(p, out, p->cap_stream);
    p->capturing_prof = false;
    g.recs.swap(p->pending);
    p->pending.swap(outside);
    cudaGraph_t cg = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(p->cap_stream, &cg);
    if (s == XEB_OK && ec != cudaSuccess)
        s = fail(XEB_ECUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(ec));
    if (s == XEB_OK) {
        const cudaError_t ei = cudaGraphInstantiate(&g.exec, cg, 0);
        if (ei != cudaSuccess) {
            g.exec = nullptr;
            s = fail(XEB_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ei));
        }
    }
    if (cg) cudaGraphDestroy(cg);
    if (s != XEB_OK) {
        drop_graph(p, g);
        return s;
    }
    g.out = out;
    return XEB_OK;
}
}  // namespace

extern "C" xeb_status xeb_amplitudes(xeb_plan_s* p, double* out_dev, uintptr_t stream) {
    xeb_status s = check_bound(p);
    if (s != XEB_OK) return s;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    double2* out = out_dev ? reinterpret_cast<double2*>(out_dev)
                           : reinterpret_cast<double2*>(p->ws + p->off_tables + p->t_amps);
    const bool use_graph = p->opts.reserved[2] == 0 && p->sliced.size() <= 6;
    if (!use_graph) {
        s = enqueue_step(p, out, st);
    } else {
        xeb_plan_s::StepGraph* g = &p->graph_plain;
        if (p->profiling) {
            g = &p->graph_prof[p->graph_prof_next];
            p->graph_prof_next ^= 1;
            if (g->launched) {  // read the events of its previous launch first
                accumulate(p, g->recs);
                g->launched = false;
            }
        }
        if (!g->exec || g->out != out) s = capture_step(p, *g, out);
        if (s == XEB_OK) {
            XEB_CUDA(cudaGraphLaunch(g->exec, st));
            g->launched = p->profiling;
        }
    }
    if (s == XEB_OK) {
        p->amps_ready = true;
        p->tables_ready = true;
    }
    return s;
}

namespace {
// The first max(1, round(frac 2^S)) draws of a partial Fisher-Yates shuffle of
// 0 .. 2^S - 1 driven by splitmix64 from `seed` (see xeb_set_slice_subset);
// empty for frac >= 1 (all values).
xeb_status subset_ids(int S, double frac, uint64_t seed, std::vector<int64_t>& ids) {
    ids.clear();
    if (!(frac > 0)) return fail(XEB_EINVAL, "slice subset fraction must be > 0");
    const int64_t n = int64_t(1) << S;
    if (frac >= 1.0) return XEB_OK;
    const int64_t cnt = std::max<int64_t>(1, std::llround(frac * double(n)));
    if (cnt > (int64_t(1) << 26)) return fail(XEB_EINVAL, "slice subset above 2^26 values");
    // partial Fisher-Yates over 0..n-1 with the swapped positions kept sparse
    std::unordered_map<int64_t, int64_t> moved;
    auto at = [&](int64_t i) {
        auto it = moved.find(i);
        return it == moved.end() ? i : it->second;
    };
    uint64_t x = seed;
    for (int64_t j = 0; j < cnt; ++j) {
        x += 0x9e3779b97f4a7c15ULL;  // splitmix64
        uint64_t z = x;
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
        z ^= z >> 31;
        const int64_t r = j + int64_t(z % uint64_t(n - j));
        const int64_t vj = at(j), vr = at(r);
        moved[r] = vj;
        ids.push_back(vr);
    }
    return XEB_OK;
}
}  // namespace

extern "C" xeb_status xeb_set_slice_subset(xeb_plan_s* p, double frac, uint64_t seed, int64_t* n_chosen) {
    if (!p) return fail(XEB_EINVAL, "plan is NULL");
    std::vector<int64_t> ids;
    const xeb_status st = subset_ids(int(p->sliced.size()), frac, seed, ids);
    if (st != XEB_OK) return st;
    p->slice_all = ids.empty();
    p->slice_ids = std::move(ids);
    drop_graph(p, p->graph_plain);
    for (auto& g : p->graph_prof) drop_graph(p, g);
    if (n_chosen) *n_chosen = p->slice_all ? int64_t(1) << p->sliced.size() : int64_t(p->slice_ids.size());
    return XEB_OK;
}

extern "C" xeb_status xeb_set_slice_block(xeb_plan_s* p, double frac, uint64_t seed, int64_t lo, int64_t hi,
                                          int64_t* n_chosen) {
    if (!p) return fail(XEB_EINVAL, "plan is NULL");
    std::vector<int64_t> ids;
    const xeb_status st = subset_ids(int(p->sliced.size()), frac, seed, ids);
    if (st != XEB_OK) return st;
    const int64_t total = ids.empty() ? int64_t(1) << p->sliced.size() : int64_t(ids.size());
    if (lo < 0 || hi < lo || hi > total)
        return fail(XEB_EINVAL, "slice block [" + std::to_string(lo) + ", " + std::to_string(hi) +
                                    ") outside the " + std::to_string(total) + " slice values");
    if (hi - lo > (int64_t(1) << 26)) return fail(XEB_EINVAL, "slice block above 2^26 values");
    std::vector<int64_t> blk;
    blk.reserve(size_t(hi - lo));
    for (int64_t i = lo; i < hi; ++i) blk.push_back(ids.empty() ? i : ids[size_t(i)]);
    p->slice_all = false;
    p->slice_ids = std::move(blk);
    drop_graph(p, p->graph_plain);
    for (auto& g : p->graph_prof) drop_graph(p, g);
    if (n_chosen) *n_chosen = hi - lo;
    return XEB_OK;
}

extern "C" xeb_status xeb_plan_slice_ids(const xeb_plan_s* p, int64_t* ids) {
    if (!p || !ids) return fail(XEB_EINVAL, "plan or ids is NULL");
    if (p->slice_all) {
        const int64_t n = int64_t(1) << p->sliced.size();
        for (int64_t i = 0; i < n; ++i) ids[i] = i;
    } else {
        std::copy(p->slice_ids.begin(), p->slice_ids.end(), ids);
    }
    return XEB_OK;
}

extern "C" xeb_status xeb_fidelity(xeb_plan_s* p, double* F, double* m1, double* m2, uintptr_t stream) {
    xeb_status s = check_bound(p);
    if (s != XEB_OK) return s;
    if (!p->amps_ready) return fail(XEB_EINVAL, "no amplitudes computed yet");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    char* tables = p->ws + p->off_tables;
    double res[4];
    int32_t err = 0;
    XEB_CUDA(cudaMemcpyAsync(res, tables + p->t_result, 32, cudaMemcpyDeviceToHost, st));
    XEB_CUDA(cudaMemcpyAsync(&err, tables + p->t_err, 4, cudaMemcpyDeviceToHost, st));
    XEB_CUDA(cudaStreamSynchronize(st));
    if (err) {   // reported once: the word is cleared so the plan's next step starts clean
        XEB_CUDA(cudaMemsetAsync(tables + p->t_err, 0, 4, st));
        XEB_CUDA(cudaStreamSynchronize(st));
    }
    if (err & xebk::kErrTimeout)
        return fail(XEB_ETIMEOUT, "a bounded device wait gave up (role " + std::to_string(err & 0xff) + ")");
    if (err) return fail(XEB_EDEVICE, "device key tables disagree with the plan's counts (node " +
                                           std::to_string(err - 1) + ")");
    if (F) *F = res[0];
    if (m1) *m1 = res[1];
    if (m2) *m2 = res[2];
    return XEB_OK;
}

// Streamed evaluation in the lexicographic order of Alg. 4: the bitstrings
// are sorted by their bits read in the tree's order pi (first bit most
// significant), so consecutive ones share the longest key prefixes, and are
// evaluated `chunk` at a time with one tree and slice set; every chunk's
// plan binds the same library workspace, grown to the largest chunk's need.
// The key tables and the arena then scale with the chunk, not with k.  A
// prefix that straddles two chunks is contracted once in each.
extern "C" xeb_status xeb_run_chunked(const xeb_circuit* circuit, const uint64_t* bits_host, size_t k,
                                      const xeb_tree* tree, const xeb_slices* slices, const xeb_plan_opts* opts,
                                      size_t chunk, double* amps_host, double* F_host, double* mean_2np_host,
                                      double* mean_2np_sq_host, uintptr_t stream) {
    if (!bits_host || k == 0) return fail(XEB_EINVAL, "need k >= 1 bitstrings");
    if (chunk == 0) return fail(XEB_EINVAL, "chunk must be >= 1");
    if (chunk > size_t(xebk::kMaxK)) return fail(XEB_EUNSUPPORTED, "chunk above the per-plan bitstring limit");
    if (k > size_t(UINT32_MAX)) return fail(XEB_EUNSUPPORTED, "more than 2^32 - 1 bitstrings");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    xeb_plan_opts o;
    if (opts) o = *opts;
    else xeb_default_opts(&o);
    o.reserved[2] = 1;   // each chunk's plan runs once: launch kernel by kernel, no graph capture
    // the tree and slices: given, or planned on the first `chunk` input
    // bitstrings (a sample of the set; the sorted order would skew it)
    xeb_plan_s* first = nullptr;
    const size_t k0 = std::min(chunk, k);
    xeb_status s = create_plan(circuit, bits_host, k0, 0, tree, slices, &o, &first);
    if (s != XEB_OK) return s;
    std::unique_ptr<xeb_plan_s, void (*)(xeb_plan_s*)> hold(first, xeb_plan_destroy);
    std::vector<int32_t> ch;
    for (const auto& pr : first->tree) { ch.push_back(pr[0]); ch.push_back(pr[1]); }
    const xeb_tree t_use{int(first->tree.size()), ch.data()};
    const std::vector<int32_t> sl(first->sliced.begin(), first->sliced.end());
    const xeb_slices s_use{int(sl.size()), sl.empty() ? nullptr : sl.data()};
    const std::vector<int> pi = first->an.pi;
    hold.reset();
    // Alg. 4 order: ascending key over the bits in pi order
    auto key_of = [&](uint64_t b) {
        uint64_t key = 0;
        for (int q : pi) key = (key << 1) | ((b >> q) & 1);
        return key;
    };
    std::vector<std::pair<uint64_t, uint32_t>> order(k);
    for (size_t i = 0; i < k; ++i) order[i] = {key_of(bits_host[i]), uint32_t(i)};
    std::stable_sort(order.begin(), order.end(),
                     [](const auto& x, const auto& y) { return x.first < y.first; });
    std::vector<uint64_t> cb(std::min(chunk, k));
    std::vector<double> ca(2 * std::min(chunk, k));
    void* ws = nullptr;
    size_t ws_bytes = 0;
    double sum_p = 0.0, sum_p2 = 0.0;   // of 2^n p and (2^n p)^2 over all k
    s = XEB_OK;
    for (size_t c0 = 0; c0 < k && s == XEB_OK; c0 += chunk) {
        const size_t kc = std::min(chunk, k - c0);
        for (size_t j = 0; j < kc; ++j) cb[j] = bits_host[order[c0 + j].second];
        xeb_plan_s* pc = nullptr;
        s = create_plan(circuit, cb.data(), kc, 0, &t_use, &s_use, &o, &pc);
        if (s != XEB_OK) break;
        std::unique_ptr<xeb_plan_s, void (*)(xeb_plan_s*)> hc(pc, xeb_plan_destroy);
        const size_t need = xeb_plan_device_bytes(pc);
        if (need > ws_bytes) {
            if (ws) cudaFree(ws);
            ws = nullptr;
            ws_bytes = 0;
            const cudaError_t e = cudaMalloc(&ws, need);
            if (e != cudaSuccess) { s = fail(XEB_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e)); break; }
            ws_bytes = need;
        }
        s = xeb_plan_bind(pc, ws, ws_bytes, stream);
        double m1 = 0, m2 = 0;
        if (s == XEB_OK) s = xeb_run(pc, cb.data(), kc, ca.data(), nullptr, stream);
        if (s == XEB_OK) s = xeb_fidelity(pc, nullptr, &m1, &m2, stream);
        if (s != XEB_OK) break;
        sum_p += m1 * double(kc);
        sum_p2 += m2 * double(kc);
        if (amps_host)
            for (size_t j = 0; j < kc; ++j) {
                const size_t i = order[c0 + j].second;
                amps_host[2 * i] = ca[2 * j];
                amps_host[2 * i + 1] = ca[2 * j + 1];
            }
    }
    if (ws) {
        cudaStreamSynchronize(st);
        cudaFree(ws);
    }
    if (s != XEB_OK) return s;
    if (F_host) *F_host = sum_p / double(k) - 1.0;
    if (mean_2np_host) *mean_2np_host = sum_p / double(k);
    if (mean_2np_sq_host) *mean_2np_sq_host = sum_p2 / double(k);
    return XEB_OK;
}

extern "C" xeb_status xeb_run(xeb_plan_s* p, const uint64_t* bits_host, size_t k, double* amps_host, double* F,
                              uintptr_t stream) {
    xeb_status s = check_bound(p);
    if (s != XEB_OK) return s;
    if (k != p->k) return fail(XEB_EINVAL, "k differs from the plan's k");
    if (!bits_host) return fail(XEB_EINVAL, "bitstrings pointer is NULL");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    char* tables = p->ws + p->off_tables;
    XEB_CUDA(cudaMemcpyAsync(tables + p->t_bits, bits_host, k * 8, cudaMemcpyHostToDevice, st));
    double* amps_dev = reinterpret_cast<double*>(tables + p->t_amps);
    s = xeb_amplitudes(p, amps_dev, stream);
    if (s != XEB_OK) return s;
    if (amps_host) XEB_CUDA(cudaMemcpyAsync(amps_host, amps_dev, (k << p->w) * 16, cudaMemcpyDeviceToHost, st));
    return xeb_fidelity(p, F, nullptr, nullptr, stream);
}

extern "C" xeb_status xeb_plan_keys(xeb_plan_s* p, int node, int32_t* key, int32_t* uL, int32_t* uR, uintptr_t stream) {
    xeb_status s = check_bound(p);
    if (s != XEB_OK) return s;
    if (node < 0 || node >= int(p->tree.size())) return fail(XEB_EINVAL, "node out of range");
    const int v = p->an.L + node;
    const int ti = p->trie_of_node[v];
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    char* tables = p->ws + p->off_tables;
    if (!p->tables_ready) {
        s = build_tables(p, st);
        if (s != XEB_OK) return s;
    }
    if (ti < 0) {  // no output bits: a single key
        if (key) std::fill(key, key + p->k, 0);
        if (uL) uL[0] = 0;
        if (uR) uR[0] = 0;
        return XEB_OK;
    }
    const xebk::TrieDesc& d = p->trie[ti];
    if (key) XEB_CUDA(cudaMemcpyAsync(key, tables + d.key_off, p->k * 4, cudaMemcpyDeviceToHost, st));
    if (uL) XEB_CUDA(cudaMemcpyAsync(uL, tables + d.uL_off, size_t(d.kv) * 4, cudaMemcpyDeviceToHost, st));
    if (uR) XEB_CUDA(cudaMemcpyAsync(uR, tables + d.uR_off, size_t(d.kv) * 4, cudaMemcpyDeviceToHost, st));
    XEB_CUDA(cudaStreamSynchronize(st));
    return XEB_OK;
}

// Autotuner: time every distinct kernel form of every contraction on the
// plan's own operands (filled by one step), keep the fastest.
extern "C" xeb_status xeb_plan_autotune(xeb_plan_s* p, int reps, uintptr_t stream, int32_t* n_changed) {
    xeb_status s = check_bound(p);
    if (s != XEB_OK) return s;
    if (reps < 1) return fail(XEB_EINVAL, "reps < 1");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const Program& pr = p->prog;
    if (p->choice.size() != pr.ops.size()) p->choice.assign(pr.ops.size(), CH_AUTO);
    const bool was_prof = p->profiling;
    p->profiling = false;
    double2* amps = reinterpret_cast<double2*>(p->ws + p->off_tables + p->t_amps);
    s = enqueue_step(p, amps, st);   // operands with realistic contents
    p->profiling = was_prof;
    if (s != XEB_OK) return s;
    XEB_CUDA(cudaStreamSynchronize(st));
    char* tables = p->ws + p->off_tables;
    cudaEvent_t e0, e1;
    XEB_CUDA(cudaEventCreate(&e0));
    XEB_CUDA(cudaEventCreate(&e1));
    int changed = 0;
    std::string why;
    for (size_t i = 0; i < pr.ops.size() && s == XEB_OK; ++i) {
        if (pr.ops[i].kind == OP_PERM || p->op_folded[i]) continue;
        const GemmLaunch keep = p->gemms[i];
        std::vector<std::pair<float, int>> timed;
        std::vector<std::pair<int, int>> seen;
        for (int ch = 0; ch < CH_COUNT && s == XEB_OK; ++ch) {
            GemmLaunch g = keep;
            if (!select_kernel(p, pr.ops[i], ch, g)) continue;
            const std::pair<int, int> form{g.kernel, g.kernel == GK_TC2             ? g.tc.tma + 2 * g.tc.grp
                                                     : g.kernel == xebk::GK_KEYED  ? g.rpt
                                                     : g.kernel == xebk::GK_STREAM ? g.s.npt * 4096 + g.s.R
                                                                                   : 0};
            if (std::find(seen.begin(), seen.end(), form) != seen.end()) continue;
            seen.push_back(form);
            p->gemms[i] = g;
            if (!validate_launches(p, why)) continue;
            auto launch = [&]() {
                return p->elem == 8 ? launch_gemm_op<float2>(p, g, reinterpret_cast<float2*>(p->ws + p->off_arena), tables, st)
                                    : launch_gemm_op<double2>(p, g, reinterpret_cast<double2*>(p->ws + p->off_arena), tables, st);
            };
            cudaError_t e = launch();   // warm-up
            if (e == cudaSuccess) e = cudaEventRecord(e0, st);
            for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch();
            if (e == cudaSuccess) e = cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) s = fail(XEB_ECUDA, std::string("autotune: ") + cudaGetErrorString(e));
            else timed.push_back({ms, ch});
        }
        p->gemms[i] = keep;
        if (s != XEB_OK || timed.size() < 2) continue;
        const auto best = *std::min_element(timed.begin(), timed.end());
        GemmLaunch g = keep;
        select_kernel(p, pr.ops[i], best.second, g);
        const bool differs = g.kernel != keep.kernel || (g.kernel == GK_TC2 && (g.tc.tma != keep.tc.tma || g.tc.grp != keep.tc.grp)) ||
                             (g.kernel == xebk::GK_KEYED && g.rpt != keep.rpt) ||
                             (g.kernel == xebk::GK_STREAM && (g.s.npt != keep.s.npt || g.s.R != keep.s.R));
        p->choice[i] = best.second;
        p->gemms[i] = g;
        changed += differs;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s == XEB_OK && !validate_launches(p, why)) s = fail(XEB_EINVAL, "autotuned launches failed validation: " + why);
    drop_graph(p, p->graph_plain);   // recaptured with the new forms
    for (auto& g : p->graph_prof) drop_graph(p, g);
    if (n_changed) *n_changed = changed;
    return s;
}

extern "C" xeb_status xeb_plan_test_wait(xeb_plan_s* p, int enable) {
    if (!p) return fail(XEB_EINVAL, "NULL plan");
    p->test_wait = enable != 0;
    for (GemmLaunch& g : p->gemms) {
        if (g.kernel == GK_TC2) g.tc.test_wait = p->test_wait;
        if (g.kernel == GK_TCKD) g.kd.test_wait = p->test_wait;
    }
    drop_graph(p, p->graph_plain);
    for (auto& g : p->graph_prof) drop_graph(p, g);
    return XEB_OK;
}

extern "C" xeb_status xeb_plan_profile(xeb_plan_s* p, int enable) {
    if (!p) return fail(XEB_EINVAL, "NULL plan");
    drain_profile(p);
    for (int c = 0; c < XEB_N_KC; ++c) p->prof_ms[c] = p->prof_n[c] = p->prof_flops[c] = p->prof_bytes[c] = 0;
    p->op_ms.clear();
    p->op_n.clear();
    p->profiling = enable != 0;
    return XEB_OK;
}

extern "C" xeb_status xeb_plan_buffers(const xeb_plan_s* p, int64_t* off, int64_t* elems, uint32_t* mask,
                                       int32_t* n_nodes) {
    if (!p || !n_nodes) return fail(XEB_EINVAL, "NULL plan or n_nodes");
    const int N = int(p->an.nodes.size());
    *n_nodes = N;
    for (int v = 0; v < N; ++v) {
        const Buffer& b = p->prog.bufs[size_t(p->prog.node_buf[size_t(v)])];
        if (off) off[v] = b.off;
        if (elems) elems[v] = b.elems;
        if (mask) mask[v] = p->node_mask[size_t(v)];
    }
    return XEB_OK;
}

extern "C" xeb_status xeb_plan_step_flops(const xeb_plan_s* p, double* flops, double* contractions) {
    if (!p) return fail(XEB_EINVAL, "NULL plan");
    const int S = int(p->sliced.size());
    const int64_t n_run = p->slice_all ? int64_t(1) << S : int64_t(p->slice_ids.size());
    double fl = 0, nc = 0;
    for (size_t i = 0; i < p->prog.ops.size(); ++i) {
        const Op& op = p->prog.ops[i];
        if (op.kind != OP_GEMM || p->op_folded[i]) continue;
        const uint32_t e = p->node_mask[size_t(op.node)];
        double times = 0;
        if (p->slice_all) {   // counting order: bit b moves every 2^b slices
            int low = 0;
            while (low < S && !((e >> low) & 1)) ++low;
            times = low >= S ? 1.0 : std::ldexp(1.0, S - low);
        } else {
            int64_t prev = 0;
            for (int64_t si = 0; si < n_run; ++si) {
                const int64_t s = p->slice_ids[size_t(si)];
                if (si == 0 || (uint32_t(s ^ prev) & e)) times += 1;
                prev = s;
            }
        }
        fl += times * 8.0 * double(op.kv) * double(op.M) * double(op.N) * double(op.K);
        nc += times;
    }
    if (flops) *flops = fl;
    if (contractions) *contractions = nc;
    return XEB_OK;
}

extern "C" xeb_status xeb_plan_op_layout(const xeb_plan_s* p, int op_index, int32_t* out, int cap, int32_t* n_out) {
    if (!p || !n_out) return fail(XEB_EINVAL, "NULL plan or n_out");
    if (op_index < 0 || size_t(op_index) >= p->prog.ops.size()) return fail(XEB_EINVAL, "op index out of range");
    const Op& op = p->prog.ops[size_t(op_index)];
    std::vector<int32_t> v = {op.kind, op.node, op.a_node, op.b_node};
    const std::vector<int>* lists[6] = {&op.a_pos_m, &op.a_pos_k, &op.b_pos_k, &op.b_pos_n, &op.c_pos_m, &op.c_pos_n};
    for (auto* l : lists) v.push_back(int32_t(l->size()));
    for (auto* l : lists) v.insert(v.end(), l->begin(), l->end());
    *n_out = int32_t(v.size());
    if (out)
        for (int i = 0; i < std::min(cap, int(v.size())); ++i) out[i] = v[size_t(i)];
    return XEB_OK;
}

extern "C" xeb_status xeb_plan_profile_ops(xeb_plan_s* p, int cap, double* ms, double* launches, int32_t* cls,
                                           double* shape, int32_t* n_ops) {
    if (!p || !n_ops) return fail(XEB_EINVAL, "NULL plan or n_ops");
    drain_profile(p);
    const Program& pr = p->prog;
    static const int cls_of[8] = {XEB_KC_GEMM_GENERIC, XEB_KC_GEMM_TILED, XEB_KC_GEMM_GEMV, XEB_KC_GEMM_TAIL,
                                  XEB_KC_GEMM_STREAM,  XEB_KC_GEMM_MEMO,  XEB_KC_GEMM_KDEEP, XEB_KC_GEMM_KEYED};
    const int n = int(pr.ops.size());
    *n_ops = n;
    for (int i = 0; i < std::min(n, cap); ++i) {
        const Op& op = pr.ops[size_t(i)];
        if (ms) ms[i] = size_t(i) < p->op_ms.size() ? p->op_ms[size_t(i)] : 0.0;
        if (launches) launches[i] = size_t(i) < p->op_n.size() ? p->op_n[size_t(i)] : 0.0;
        if (cls) {
            if (op.kind == OP_PERM) cls[i] = XEB_KC_PERMUTE;
            else if (!p->bound || p->gemms.size() <= size_t(i)) cls[i] = -1;
            else {
                const int kk = p->gemms[size_t(i)].kernel;
                cls[i] = kk == GK_TCKD ? XEB_KC_GEMM_TC_KDEEP : kk >= GK_TC2 ? XEB_KC_GEMM_TC : cls_of[kk];
            }
        }
        if (shape) {
            shape[4 * i + 0] = double(op.M);
            shape[4 * i + 1] = double(op.N);
            shape[4 * i + 2] = double(op.K);
            shape[4 * i + 3] = double(op.kv);
        }
    }
    return XEB_OK;
}

extern "C" xeb_status xeb_plan_op_form(const xeb_plan_s* p, int op_index, int32_t* form) {
    if (!p || !form) return fail(XEB_EINVAL, "NULL plan or form");
    if (!p->bound) return fail(XEB_EINVAL, "plan not bound to device memory (call xeb_plan_bind)");
    if (op_index < 0 || size_t(op_index) >= p->prog.ops.size() || p->prog.ops[size_t(op_index)].kind == OP_PERM ||
        p->gemms.size() <= size_t(op_index))
        return fail(XEB_EINVAL, "op_index is not a contraction step of the plan");
    static const int cls_of[8] = {XEB_KC_GEMM_GENERIC, XEB_KC_GEMM_TILED, XEB_KC_GEMM_GEMV, XEB_KC_GEMM_TAIL,
                                  XEB_KC_GEMM_STREAM,  XEB_KC_GEMM_MEMO,  XEB_KC_GEMM_KDEEP, XEB_KC_GEMM_KEYED};
    const GemmLaunch& g = p->gemms[size_t(op_index)];
    const int kk = g.kernel;
    form[0] = kk == GK_TCKD ? XEB_KC_GEMM_TC_KDEEP : kk >= GK_TC2 ? XEB_KC_GEMM_TC : cls_of[kk];
    form[1] = kk == xebk::GK_KEYED ? g.rpt : 0;
    form[2] = kk == xebk::GK_STREAM || kk == xebk::GK_MEMO ? g.s.npt : 0;
    form[3] = kk == xebk::GK_STREAM || kk == xebk::GK_MEMO ? g.s.R : 0;
    form[4] = kk == GK_TC2 ? g.tc.tma : 0;
    return XEB_OK;
}

extern "C" xeb_status xeb_plan_profile_read(xeb_plan_s* p, double* ms, double* n, double* flops, double* bytes) {
    if (!p) return fail(XEB_EINVAL, "NULL plan");
    drain_profile(p);
    for (int c = 0; c < XEB_N_KC; ++c) {
        if (ms) ms[c] = p->prof_ms[c];
        if (n) n[c] = p->prof_n[c];
        if (flops) flops[c] = p->prof_flops[c];
        if (bytes) bytes[c] = p->prof_bytes[c];
    }
    return XEB_OK;
}
