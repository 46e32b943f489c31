// Device-side descriptors and launch wrappers of the contraction kernels.
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

namespace xebk {

constexpr int kMaxTrieK = 16384;  // bitstrings per single-CTA key-table sort
constexpr int kMaxK = 1 << 24;     // bitstrings per plan (multi-CTA key-table sort beyond kMaxTrieK)

// Memo key table of one tree node that depends on output bits (a1).
struct TrieDesc {
    int a, b;            // range of the node's bits in pi
    int kv;              // planned number of distinct values
    int is_internal;
    int64_t key_off;     // int32 [k]   key id of every bitstring
    int64_t uniq_off;    // uint64 [kv] value of every key (ascending)
    int64_t rep_off;     // int32 [kv]  one bitstring having that key
    int64_t uL_off;      // int32 [kv]  left child's key id (internal)
    int64_t uR_off;      // int32 [kv]  right child's key id (internal)
    int64_t gstart_off;  // int32 [kL+1] first key of every left-key group (internal)
    int64_t l_key_off;   // left child's key array, -1 if the child has no bits
    int64_t r_key_off;   // right child's key array, -1 if the child has no bits
    int kL;              // left child's key count
    int pad;
};

// Leaf materialisation (a2): projected leaf tensor per key and slice.
struct LeafDesc {
    int64_t dst_off;     // element offset in the arena
    int64_t src_off;     // element offset in the leaf data
    int r;               // stored rank (bond legs not sliced)
    int n_out;           // output bits of the leaf
    int n_canon;         // canonical rank = n_out + all bond legs (sliced too)
    int kv;
    int src_pos[8];      // stored bit j (0 = fastest) -> canonical bit position
    int n_sl;
    int sl_pos[4];       // canonical bit position of the leaf's sliced legs
    int sl_bit[4];       // their bit in the slice index
    int64_t uniq_off;    // trie uniq table of the leaf (-1 if no output bits)
};

// Tiled bit permutation (a3): dst bit j <- src bit perm[j].
struct PermDesc {
    int r, u, n_outer;
    int usrc[12];        // tile bit i (src order) -> src bit position
    int udst_e[12];      // dst-order tile bit i -> src-order tile bit
    int udst[12];        // dst-order tile bit i -> dst bit position
    int outer_src[48];   // outer bit i -> src bit position
    int outer_dst[48];   // outer bit i -> dst bit position
    int64_t keys;
};

// One pairwise contraction, for u < kv: C_u = A_{uL(u)} (M x K) * B_{uR(u)} (K x N).
// Operands are read in place: bit i of the row index m sits at address bit
// apm[i] of A's tensor, bit i of the summed index k at apk[i] (A) / bpk[i] (B),
// bit i of the column index n at bpn[i] (B).  C is written row-major [M][N].
constexpr int kMaxLegs = 48;
struct GemmDesc {
    int64_t M, N, K, kv;
    int64_t a_off, a_key, b_off, b_key, c_off, c_key;
    int nam, nak, nbk, nbn;
    int8_t apm[kMaxLegs], apk[kMaxLegs], bpk[kMaxLegs], bpn[kMaxLegs];
    int8_t cpm[kMaxLegs], cpn[kMaxLegs];  // result address bit of m bit i / n bit i
    int c_natural;                        // 1: result is row-major [M][N]
    const int32_t* uL;      // nullptr -> 0
    const int32_t* uR;      // nullptr -> 0
    const int32_t* gstart;  // groups of keys by uL (nullptr -> one group)
    int64_t n_groups;
};

// Streaming tile of the memory-bound contraction kernel: R rows x all K of A
// occupy tile index bits 0..T-1 in ascending address order; tile bit i sits
// at address bit pos[i] and is a bit of k if (is_k >> i) & 1, else of r.
struct StreamDesc {
    int R, tm, T, npt;
    uint32_t is_k;
    int8_t pos[32];
};

enum GemmKernel { GK_GENERIC = 0, GK_TILED = 1, GK_GEMV = 2, GK_TAIL = 3, GK_STREAM = 4, GK_MEMO = 5, GK_KDEEP = 6,
                  GK_KEYED = 7 };
constexpr int kKdTile = 32;   // deep-K contractions: 32 x 32 result tile per CTA
constexpr int kKdChunk = 64;  // summed-index chunk staged per step (8 per warp)
constexpr int kStreamMaxK = 64, kStreamMaxN = 64;
constexpr int kStreamEPT = 8;   // A-tile elements per thread
constexpr int kStreamStages = 4;  // A tiles in flight per CTA
constexpr int kStreamBKeys = 2048;  // B elements staged per key batch (N == 1)
constexpr int kMemoBPre = 512;      // memo levels: B elements loaded with each tile (one left-key group)

// tcgen05 split-precision contraction (one key, M % 128 == 0, 16 <= K, N <= 64).
// Tile bits of one K-chunk: the 7 lowest row bits and the 4 lowest summed
// bits, in ascending address order (pos / is_k as in StreamDesc); the
// remaining summed bits select the chunk (chunk_off).
struct TcDesc {
    int64_t M;
    int K2, N2, n_chunks, tmem_cols;
    int64_t a_off, b_off, c_off;
    int nam, nbk, nbn, T;
    uint32_t is_k;
    int8_t apm[kMaxLegs], bpk[kMaxLegs], bpn[kMaxLegs];
    int8_t pos[16];
    int32_t chunk_off[4];
    // (tensor-memory variant) rows outside the tile: A and C address bits;
    // the result tile's bits in ascending C address: C bit, is-column flag
    // and the row / column bit index
    int n_ext;
    int8_t ext_apos[kMaxLegs], ext_cpos[kMaxLegs];
    int Tst;
    uint32_t st_is_n;
    int8_t st_pos[16], st_idx[16];
    // staging swizzle of the result tile (tensor-memory variant): element
    // (row, n) of the tile is staged at float2 slot row * 64 + (n ^ x), where
    // x is the XOR of st_swz[i] over the tile bits i (ascending C address
    // order) set in (row, n); st_swz[i] < 16 and is 0 for column bits below 4
    int8_t st_swz[16];
    int32_t* err;         // error word (timeouts)
    // split of the operands (see tc_gemm2.cu): big parts on a common grid of
    // 2^split_bits units per state row and chunk / per W^T row; split_terms =
    // 3 (big*big, big*small, small*big) or 4 (+ small*small)
    int split_bits, split_terms;
    uint64_t wait_ns;     // limit of every device-side wait (ns of %globaltimer)
    int test_wait;        // testing aid: the MMA thread first waits on a barrier nothing completes
    // (tensor-memory variant, TMA mode) A is a row-major [M][K] matrix; a
    // chunk is 2^(kTc2RowBits - box_log2) boxes of 32 floats x 2^box_log2
    // consecutive rows; box j starts box_y[j] rows above the tile's base row,
    // and an outside-tile A address bit p is row bit p - row_shift
    int tma, box_log2, row_shift;
    int32_t box_y[16];
    // (tensor-memory variant, gather mode) grouped mode for memo-trie levels:
    // tiles g * tpg .. (g + 1) * tpg - 1 belong to left-key group g, whose A
    // starts grp_a[g] elements after a_off and whose keys gstart[g] ..
    // gstart[g + 1] - 1 form the columns: key u's B vector (K complex) sits at
    // bpack_off + u K and its results at c_off + u c_key + row
    int grp;
    int64_t tpg, n_groups, c_key, bpack_off;
    const int32_t* gstart;
    const int64_t* grp_a;
    // (grouped instantiation) keyed mode: one group per key u of a keyed
    // contraction C_u = A_uL(u) B_uR(u); A at a_off + uL[u] a_key, B at b_off +
    // uR[u] b_key (W^T rewritten when the key changes), C at c_off + u c_key;
    // each CTA takes a contiguous block of tiles
    int keyed;
    int64_t a_key, b_key;
    const int32_t* uL;
    const int32_t* uR;
};
// tcgen05 split-precision form of keyed contractions with a deep summed
// index (tc_kdeep.cu): C_u = A_uL(u) (M x K) B_uR(u) (K x N) for every key u,
// M, N in {16, 32}, K a multiple of 64 complex.  Operand
// addressing as in GemmDesc (bit i of m / k / n at address bit apm / apk /
// bpk / bpn [i] of the key's block; result bit i of m / n at cpm / cpn [i]).
struct KdDesc {
    int64_t a_off, a_key, b_off, b_key, c_off, c_key;
    const int32_t* uL;
    const int32_t* uR;
    const int32_t* gstart;
    int64_t n_groups, kv;
    int M, N, K, nak, nbk;   // M, N in {16, 32}
    int8_t apm[5], bpn[5], cpm[5], cpn[5];
    int8_t apk[kMaxLegs], bpk[kMaxLegs];
    int32_t* err;
    int split_bits, split_terms, test_wait;
    uint64_t wait_ns;
};
cudaError_t launch_tc_kdeep(const KdDesc& d, float2* arena, int n_sms, cudaStream_t st);
// Keyed contractions with K in {4, 8, 16, 32}, N in {1, 2, 4, 8, 16} complex,
// M >= 32 a multiple of 32, row-major results, keys grouped by left key
// (keyed.cu, complex64).  Scratch: keyed_scratch_bytes(kvB, K, N) bytes,
// 256-byte aligned, for the packed copy of the kvB right operands.
// rows_per_lane = 2: each lane takes two rows 32 apart (items of 64 rows,
// M % 64 == 0, K <= 16), so each uniform load of B feeds twice the
// multiply-adds.
bool keyed_fits(int64_t M, int64_t N, int64_t K);
bool keyed_fits_rows2(int64_t M, int64_t N, int64_t K);
size_t keyed_scratch_bytes(int64_t kvB, int64_t K, int64_t N);
cudaError_t launch_gemm_keyed(const GemmDesc& g, int64_t kvB, int rows_per_lane, float2* arena, char* scratch,
                              int n_sms, cudaStream_t st);

constexpr int32_t kErrTimeout = 0x40000000;  // | role code
constexpr int kTc2RowBits = 7;               // tensor-memory variant: 128 state rows per tile

// ---- launch wrappers (all asynchronous on `st`) --------------------------------
// Raise the dynamic shared-memory limits of every kernel (once per process,
// before any stream capture).
cudaError_t prepare_kernels();
cudaError_t launch_trie_keys(const TrieDesc* d_desc, int n_nodes, const uint64_t* bits, int k,
                             const int32_t* pi, char* tables, int32_t* err, cudaStream_t st);
// a1 for k > kMaxTrieK: scratch of trie_sort_scratch_bytes(k) bytes (256-byte
// aligned); h_desc = host copy of the node descriptors
size_t trie_sort_scratch_bytes(int k);
cudaError_t launch_trie_keys_large(const TrieDesc* d_desc, const TrieDesc* h_desc, int n_nodes,
                                   const uint64_t* bits, int k, const int32_t* pi, char* tables, char* scratch,
                                   int32_t* err, cudaStream_t st);
cudaError_t launch_trie_links(const TrieDesc* d_desc, const int* d_internal, int n_internal,
                              int max_kv, char* tables, cudaStream_t st);
template <typename T>
cudaError_t launch_leaves(const LeafDesc* d_desc, int n_leaves, const T* leafdata, T* arena,
                          const char* tables, int64_t slice, cudaStream_t st);
template <typename T>
cudaError_t launch_permute(const PermDesc& p, const T* src, T* dst, cudaStream_t st);
template <typename T>
cudaError_t launch_gemm(int kernel, const GemmDesc& g, T* arena, cudaStream_t st);
template <typename T>
cudaError_t launch_gemm_stream(const GemmDesc& g, const StreamDesc& s, T* arena, cudaStream_t st);
// memo-trie levels (N = 1, keys grouped by uL): scratch of memo_scratch_bytes
// for the per-group A offsets and the packed B vectors
size_t memo_scratch_bytes(int64_t n_groups, int64_t kv, int64_t K, size_t elem);
template <typename T>
cudaError_t launch_gemm_memo(const GemmDesc& g, const StreamDesc& s, T* arena, char* scratch, cudaStream_t st);
// the memo-level prep alone (per-group A offsets, packed B vectors), for the
// grouped tensor-core path
template <typename T>
cudaError_t launch_memo_prep(const GemmDesc& g, T* arena, char* scratch, cudaStream_t st);
template <typename T>
cudaError_t launch_root_accum(const T* root, double2* acc, int64_t kv, cudaStream_t st);
// tcgen05 split-precision contraction with W^T in tensor memory (128-row
// tiles, tile bits = 7 row bits + 4 k bits); tmap: 2-D tensor map of A (used
// when t.tma != 0)
cudaError_t launch_tc_gemm2(const TcDesc& t, const CUtensorMap& tmap, float2* arena, int n_sms, cudaStream_t st);
// Multi-batch plans: the root tensor of each key holds 2^w values, one per
// value x of the open qubits; bit j of x (open qubits in ascending order)
// sits at address bit pos[j] of the root's block.  w = 0: one value per key.
struct RootMap {
    int w;
    int8_t pos[16];
};
cudaError_t launch_gather_xeb(const double2* acc, const int32_t* key_root, int64_t k, const RootMap& rm,
                              double2* amps, double* partials, int n_blocks, double* result,
                              int n_qubits, cudaStream_t st);

}  // namespace xebk
