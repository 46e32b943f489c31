// CUDA kernels of the memoized multi-amplitude contraction (sm_103a).
//
//  a1  k_trie_keys / k_trie_links : memo key tables.  A subexpression is
//      evaluated once per distinct value of its variables (Sec. "Multi-tensor
//      contraction algorithm"); keys are ranks of the node's output-bit range
//      read as a number, i.e. the lexicographic order of App. C (Alg. 3).
//  a2  k_leaves      : leaf tensors projected on output bits and sliced legs.
//  a3  k_permute     : leg permutation of complex tensors (legs have dim 2, so
//      a permutation of the index bits), tiled through shared memory so both
//      the reads and the writes are contiguous runs.
//  a4  k_gemm_*      : the pairwise contraction T*S of Eq. (elem-cont) as one
//      complex GEMM per key, C_u = A_{uL(u)} B_{uR(u)}, FP32 (or FP64) FMA.
//  a5  k_gemm_tail   : tiny near-root contractions, a warp per key with a
//      shuffle reduction.
//  a6  k_root_accum  : FP64 accumulation of the root over slices (Sec.
//      "Slicing": contract per value of the fixed legs, then sum).
//  a7  k_gather_xeb / k_xeb_final : amplitudes in input order and the linear
//      XEB F = 2^n/k sum_i p(s_i) - 1 of Eq. (1), FP64, fixed reduction order.
#include "kernels.cuh"

#include <utility>

namespace xebk {

// ---- complex helpers -----------------------------------------------------------
__device__ __forceinline__ float2 cfma(float2 acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
    return acc;
}
__device__ __forceinline__ double2 cfma(double2 acc, double2 a, double2 b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
    return acc;
}
template <typename T> __device__ __forceinline__ T czero();
template <> __device__ __forceinline__ float2 czero<float2>() { return make_float2(0.f, 0.f); }
template <> __device__ __forceinline__ double2 czero<double2>() { return make_double2(0.0, 0.0); }
__device__ __forceinline__ float2 shfl_down(float2 v, int d) {
    v.x = __shfl_down_sync(0xffffffffu, v.x, d);
    v.y = __shfl_down_sync(0xffffffffu, v.y, d);
    return v;
}
__device__ __forceinline__ double2 shfl_down(double2 v, int d) {
    v.x = __shfl_down_sync(0xffffffffu, v.x, d);
    v.y = __shfl_down_sync(0xffffffffu, v.y, d);
    return v;
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

static inline int grid_for(int64_t work, int per_block, int cap) {
    int64_t b = (work + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return int(b);
}

// ---- a1: memo key tables ---------------------------------------------------------

// Block-wide exclusive scan of one int per thread (blockDim.x <= 1024).
__device__ int block_exclusive_scan(int v, int* total) {
    __shared__ int warp_tot[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
    for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        int t = lane < nw ? warp_tot[lane] : 0;
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, d);
            if (lane >= d) t += y;
        }
        warp_tot[lane] = t;  // inclusive
    }
    __syncthreads();
    const int before = wid > 0 ? warp_tot[wid - 1] : 0;
    *total = warp_tot[((blockDim.x + 31) >> 5) - 1];
    __syncthreads();
    return before + x - v;
}

__global__ void __launch_bounds__(1024) k_trie_keys(const TrieDesc* desc, const uint64_t* bits, int k,
                                                     int kpad, const int32_t* pi, char* tables,
                                                     int32_t* err) {
    extern __shared__ uint64_t sm_trie[];
    uint64_t* val = sm_trie;
    int32_t* idx = reinterpret_cast<int32_t*>(sm_trie + kpad);
    const TrieDesc d = desc[blockIdx.x];
    for (int i = threadIdx.x; i < kpad; i += blockDim.x) {
        if (i < k) {
            const uint64_t s = bits[i];
            uint64_t v = 0;
            for (int t = d.a; t < d.b; ++t) v = (v << 1) | ((s >> pi[t]) & 1ull);
            val[i] = v;
            idx[i] = i;
        } else {
            val[i] = ~0ull;
            idx[i] = 0x7fffffff;
        }
    }
    __syncthreads();
    // bitonic sort of (val, idx) ascending
    for (int size = 2; size <= kpad; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < (kpad >> 1); t += blockDim.x) {
                const int i = 2 * t - (t & (stride - 1));
                const int j = i + stride;
                const bool up = (i & size) == 0;
                const uint64_t vi = val[i], vj = val[j];
                const int32_t ii = idx[i], ij = idx[j];
                const bool gt = vi > vj || (vi == vj && ii > ij);
                if (gt == up) {
                    val[i] = vj; val[j] = vi;
                    idx[i] = ij; idx[j] = ii;
                }
            }
            __syncthreads();
        }
    }
    // ranks of distinct values
    const int chunk = (k + blockDim.x - 1) / blockDim.x;
    const int lo = threadIdx.x * chunk;
    const int hi = min(k, lo + chunk);
    int cnt = 0;
    for (int i = lo; i < hi; ++i) cnt += (i == 0 || val[i] != val[i - 1]);
    int total = 0;
    int rank = block_exclusive_scan(cnt, &total) - 1;
    int32_t* key = reinterpret_cast<int32_t*>(tables + d.key_off);
    uint64_t* uniq = reinterpret_cast<uint64_t*>(tables + d.uniq_off);
    int32_t* rep = reinterpret_cast<int32_t*>(tables + d.rep_off);
    for (int i = lo; i < hi; ++i) {
        if (i == 0 || val[i] != val[i - 1]) {
            ++rank;
            if (rank < d.kv) {
                uniq[rank] = val[i];
                rep[rank] = idx[i];
            }
        }
        key[idx[i]] = min(rank, d.kv - 1);  // ids stay inside planned tables
    }
    for (int r = total + threadIdx.x; r < d.kv; r += blockDim.x) {  // count mismatch: keep tables valid
        uniq[r] = 0;
        rep[r] = 0;
    }
    if (threadIdx.x == 0 && total != d.kv) atomicExch(err, 1 + int(blockIdx.x));
}

__global__ void k_trie_links(const TrieDesc* desc, const int* internal, char* tables) {
    const TrieDesc d = desc[internal[blockIdx.y]];
    const int32_t* rep = reinterpret_cast<const int32_t*>(tables + d.rep_off);
    const int32_t* lk = d.l_key_off >= 0 ? reinterpret_cast<const int32_t*>(tables + d.l_key_off) : nullptr;
    const int32_t* rk = d.r_key_off >= 0 ? reinterpret_cast<const int32_t*>(tables + d.r_key_off) : nullptr;
    int32_t* uL = reinterpret_cast<int32_t*>(tables + d.uL_off);
    int32_t* uR = reinterpret_cast<int32_t*>(tables + d.uR_off);
    int32_t* gs = reinterpret_cast<int32_t*>(tables + d.gstart_off);
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < d.kv; u += gridDim.x * blockDim.x) {
        const int rp = rep[u];
        const int l = lk ? lk[rp] : 0;
        const int r = rk ? rk[rp] : 0;
        uL[u] = l;
        uR[u] = r;
        const int lprev = u > 0 ? (lk ? lk[rep[u - 1]] : 0) : -1;
        if (u == 0 || l != lprev) gs[l] = u;
        if (u == d.kv - 1) gs[d.kL] = d.kv;
    }
}

cudaError_t launch_trie_keys(const TrieDesc* d_desc, int n_nodes, const uint64_t* bits, int k,
                             const int32_t* pi, char* tables, int32_t* err, cudaStream_t st) {
    if (n_nodes == 0) return cudaSuccess;
    int kpad = 2;
    while (kpad < k) kpad <<= 1;
    const size_t smem = size_t(kpad) * (sizeof(uint64_t) + sizeof(int32_t));
    k_trie_keys<<<n_nodes, 1024, smem, st>>>(d_desc, bits, k, kpad, pi, tables, err);
    return cudaGetLastError();
}

// ---- a1 for large k: one LSD radix sort per node across CTAs ----------------------
// Same tables as k_trie_keys (keys are ranks of the node's bit-range value),
// for k beyond one CTA's shared memory.  Per 8-bit digit: a per-tile
// histogram, one scan of (digit, tile) counts, and a stable scatter that ranks
// equal digits within a warp with __match_any_sync and across warps with
// per-warp digit counts; then run boundaries are counted per tile, scanned,
// and every bitstring gets the rank of its run.
constexpr int kRsThreads = 256;
constexpr int kRsTile = 4096;   // elements per CTA tile

__global__ void __launch_bounds__(kRsThreads) k_rs_extract(const TrieDesc* desc, int node, const uint64_t* bits,
                                                           int k, const int32_t* pi, uint64_t* keys, int32_t* vals) {
    const int a = desc[node].a, b = desc[node].b;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) {
        const uint64_t s = bits[i];
        uint64_t v = 0;
        for (int t = a; t < b; ++t) v = (v << 1) | ((s >> pi[t]) & 1ull);
        keys[i] = v;
        vals[i] = i;
    }
}

__global__ void __launch_bounds__(kRsThreads) k_rs_hist(const uint64_t* keys, int k, int shift, int32_t* hist,
                                                        int nb) {
    __shared__ int32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int base = blockIdx.x * kRsTile;
    for (int j = threadIdx.x; j < kRsTile; j += kRsThreads) {
        const int i = base + j;
        if (i < k) atomicAdd(&h[int((keys[i] >> shift) & 255u)], 1);
    }
    __syncthreads();
    hist[threadIdx.x * nb + blockIdx.x] = h[threadIdx.x];  // digit-major: scan gives stable bucket starts
}

// exclusive scan of n int32 in place, one CTA
__global__ void __launch_bounds__(1024) k_rs_scan(int32_t* a, int n) {
    const int chunk = (n + blockDim.x - 1) / blockDim.x;
    const int lo = min(n, int(threadIdx.x) * chunk), hi = min(n, lo + chunk);
    int sum = 0;
    for (int i = lo; i < hi; ++i) sum += a[i];
    int total = 0;
    int run = block_exclusive_scan(sum, &total);
    for (int i = lo; i < hi; ++i) {
        const int v = a[i];
        a[i] = run;
        run += v;
    }
}

__global__ void __launch_bounds__(kRsThreads) k_rs_scatter(const uint64_t* kin, const int32_t* vin, uint64_t* kout,
                                                           int32_t* vout, int k, int shift, const int32_t* off,
                                                           int nb) {
    __shared__ int32_t run[256];
    __shared__ int32_t wcnt[kRsThreads / 32][256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    run[threadIdx.x] = off[threadIdx.x * nb + blockIdx.x];
    const int base = blockIdx.x * kRsTile;
    for (int r = 0; r < kRsTile / kRsThreads; ++r) {
        for (int j = threadIdx.x; j < (kRsThreads / 32) * 256; j += kRsThreads) (&wcnt[0][0])[j] = 0;
        __syncthreads();
        const int i = base + r * kRsThreads + threadIdx.x;   // elements in order: stable
        const bool live = i < k;
        const uint64_t key = live ? kin[i] : 0;
        const int32_t val = live ? vin[i] : 0;
        const int dg = live ? int((key >> shift) & 255u) : 256 + lane;   // dead lanes: unique non-digits
        const unsigned same = __match_any_sync(0xffffffffu, dg);
        const int rank_w = __popc(same & ((1u << lane) - 1u));
        if (live && rank_w == 0) wcnt[w][dg] = __popc(same);
        __syncthreads();
        if (live) {
            int pre = 0;
            for (int ww = 0; ww < w; ++ww) pre += wcnt[ww][dg];
            const int pos = run[dg] + pre + rank_w;
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
        int add = 0;
        for (int ww = 0; ww < kRsThreads / 32; ++ww) add += wcnt[ww][threadIdx.x];
        run[threadIdx.x] += add;
        __syncthreads();
    }
}

// number of run starts (key differs from its predecessor) per tile
__global__ void __launch_bounds__(kRsThreads) k_rs_flags(const uint64_t* keys, int k, int32_t* cnt) {
    const int base = blockIdx.x * kRsTile;
    int c = 0;
    for (int j = threadIdx.x; j < kRsTile; j += kRsThreads) {
        const int i = base + j;
        if (i < k && (i == 0 || keys[i] != keys[i - 1])) ++c;
    }
    int total = 0;
    block_exclusive_scan(c, &total);
    if (threadIdx.x == 0) cnt[blockIdx.x] = total;
}

// ranks: every bitstring gets the rank of its run; run starts write the
// distinct value and a representative; the node's count is checked
__global__ void __launch_bounds__(kRsThreads) k_rs_rank(const TrieDesc* desc, int node, const uint64_t* keys,
                                                        const int32_t* vals, int k, const int32_t* cnt_off,
                                                        char* tables, int32_t* err) {
    const TrieDesc d = desc[node];
    constexpr int kPer = kRsTile / kRsThreads;   // consecutive elements per thread
    const int lo = blockIdx.x * kRsTile + threadIdx.x * kPer;
    int c = 0;
    for (int j = 0; j < kPer; ++j) {
        const int i = lo + j;
        if (i < k && (i == 0 || keys[i] != keys[i - 1])) ++c;
    }
    int total = 0;
    int rank = cnt_off[blockIdx.x] + block_exclusive_scan(c, &total) - 1;
    int32_t* key = reinterpret_cast<int32_t*>(tables + d.key_off);
    uint64_t* uniq = reinterpret_cast<uint64_t*>(tables + d.uniq_off);
    int32_t* rep = reinterpret_cast<int32_t*>(tables + d.rep_off);
    for (int j = 0; j < kPer; ++j) {
        const int i = lo + j;
        if (i >= k) break;
        if (i == 0 || keys[i] != keys[i - 1]) {
            ++rank;
            if (rank < d.kv) {
                uniq[rank] = keys[i];
                rep[rank] = vals[i];
            }
        }
        key[vals[i]] = min(rank, d.kv - 1);   // ids stay inside planned tables
        if (i == k - 1) {
            if (rank + 1 != d.kv) atomicExch(err, 1 + node);
            for (int r = rank + 1; r < d.kv; ++r) {   // count mismatch: keep tables valid
                uniq[r] = 0;
                rep[r] = 0;
            }
        }
    }
}

size_t trie_sort_scratch_bytes(int k) {
    const size_t nb = size_t((k + kRsTile - 1) / kRsTile);
    return 2 * size_t(k) * 8 + 2 * size_t(k) * 4 + 256 * nb * 4 + nb * 4 + 4 * 256;
}

cudaError_t launch_trie_keys_large(const TrieDesc* d_desc, const TrieDesc* h_desc, int n_nodes,
                                   const uint64_t* bits, int k, const int32_t* pi, char* tables, char* scratch,
                                   int32_t* err, cudaStream_t st) {
    const int nb = (k + kRsTile - 1) / kRsTile;
    uint64_t* k0 = reinterpret_cast<uint64_t*>(scratch);
    uint64_t* k1 = k0 + k;
    int32_t* v0 = reinterpret_cast<int32_t*>(k1 + k);
    int32_t* v1 = v0 + k;
    int32_t* hist = v1 + k;
    int32_t* cnt = hist + 256 * nb;
    for (int node = 0; node < n_nodes; ++node) {
        const int width = h_desc[node].b - h_desc[node].a;
        k_rs_extract<<<grid_for(k, kRsThreads, 4096), kRsThreads, 0, st>>>(d_desc, node, bits, k, pi, k0, v0);
        for (int shift = 0; shift < width; shift += 8) {
            k_rs_hist<<<nb, kRsThreads, 0, st>>>(k0, k, shift, hist, nb);
            k_rs_scan<<<1, 1024, 0, st>>>(hist, 256 * nb);
            k_rs_scatter<<<nb, kRsThreads, 0, st>>>(k0, v0, k1, v1, k, shift, hist, nb);
            std::swap(k0, k1);
            std::swap(v0, v1);
        }
        k_rs_flags<<<nb, kRsThreads, 0, st>>>(k0, k, cnt);
        k_rs_scan<<<1, 1024, 0, st>>>(cnt, nb);
        k_rs_rank<<<nb, kRsThreads, 0, st>>>(d_desc, node, k0, v0, k, cnt, tables, err);
    }
    return cudaGetLastError();
}

cudaError_t launch_trie_links(const TrieDesc* d_desc, const int* d_internal, int n_internal, int max_kv,
                              char* tables, cudaStream_t st) {
    if (n_internal == 0) return cudaSuccess;
    dim3 grid(grid_for(max_kv, 256, 64), n_internal);
    k_trie_links<<<grid, 256, 0, st>>>(d_desc, d_internal, tables);
    return cudaGetLastError();
}

// ---- a2: leaves ------------------------------------------------------------------

template <typename T>
__global__ void k_leaves(const LeafDesc* desc, const T* leafdata, T* arena, const char* tables,
                         int64_t slice) {
    const LeafDesc d = desc[blockIdx.x];
    const uint64_t* uniq = d.uniq_off >= 0 ? reinterpret_cast<const uint64_t*>(tables + d.uniq_off) : nullptr;
    int64_t sl_base = 0;
    for (int t = 0; t < d.n_sl; ++t)
        if ((slice >> d.sl_bit[t]) & 1) sl_base |= int64_t(1) << d.sl_pos[t];
    const int64_t per = int64_t(1) << d.r;
    for (int64_t e = threadIdx.x; e < int64_t(d.kv) * per; e += blockDim.x) {
        const int64_t u = e >> d.r, x = e & (per - 1);
        const uint64_t v = uniq ? uniq[u] : 0;
        int64_t src = (int64_t(v) << (d.n_canon - d.n_out)) | sl_base;
        for (int j = 0; j < d.r; ++j)
            if ((x >> j) & 1) src |= int64_t(1) << d.src_pos[j];
        arena[d.dst_off + e] = leafdata[d.src_off + src];
    }
}

template <typename T>
cudaError_t launch_leaves(const LeafDesc* d_desc, int n_leaves, const T* leafdata, T* arena,
                          const char* tables, int64_t slice, cudaStream_t st) {
    if (n_leaves <= 0) return cudaSuccess;
    k_leaves<T><<<n_leaves, 128, 0, st>>>(d_desc, leafdata, arena, tables, slice);
    return cudaGetLastError();
}

// ---- a3: permutation ----------------------------------------------------------------

template <typename T>
__global__ void __launch_bounds__(256) k_permute(const PermDesc p, const T* __restrict__ src,
                                                 T* __restrict__ dst, int64_t n_tiles) {
    extern __shared__ __align__(16) unsigned char sm_perm[];
    T* tile = reinterpret_cast<T*>(sm_perm);
    const int tsz = 1 << p.u;
    for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const int64_t key = t >> p.n_outer;
        const int64_t o = t & ((int64_t(1) << p.n_outer) - 1);
        int64_t so = key << p.r, dso = key << p.r;
        for (int i = 0; i < p.n_outer; ++i)
            if ((o >> i) & 1) {
                so |= int64_t(1) << p.outer_src[i];
                dso |= int64_t(1) << p.outer_dst[i];
            }
        for (int e = threadIdx.x; e < tsz; e += blockDim.x) {
            int64_t off = so;
            for (int i = 0; i < p.u; ++i)
                if ((e >> i) & 1) off |= int64_t(1) << p.usrc[i];
            tile[e] = src[off];
        }
        __syncthreads();
        for (int f = threadIdx.x; f < tsz; f += blockDim.x) {
            int e = 0;
            int64_t off = dso;
            for (int i = 0; i < p.u; ++i)
                if ((f >> i) & 1) {
                    e |= 1 << p.udst_e[i];
                    off |= int64_t(1) << p.udst[i];
                }
            dst[off] = tile[e];
        }
        __syncthreads();
    }
}

template <typename T>
cudaError_t launch_permute(const PermDesc& p, const T* src, T* dst, cudaStream_t st) {
    const int64_t n_tiles = p.keys << p.n_outer;
    const int grid = grid_for(n_tiles, 1, 152 * 16);
    k_permute<T><<<grid, 256, sizeof(T) << p.u, st>>>(p, src, dst, n_tiles);
    return cudaGetLastError();
}

// ---- a4/a5: contractions ----------------------------------------------------------

// Address offset of index x whose bit i sits at address bit pos[i].
__device__ __forceinline__ int64_t scatter(int64_t x, const int8_t* pos, int n) {
    int64_t off = 0;
    for (int i = 0; x != 0 && i < n; ++i, x >>= 1)
        if (x & 1) off |= int64_t(1) << pos[i];
    return off;
}

template <typename T>
__global__ void k_gemm_generic(const __grid_constant__ GemmDesc g, T* __restrict__ arena) {
    const int64_t total = g.kv * g.M * g.N;
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total;
         e += int64_t(gridDim.x) * blockDim.x) {
        const int64_t n = e % g.N;
        const int64_t rest = e / g.N;
        const int64_t m = rest % g.M;
        const int64_t u = rest / g.M;
        const int64_t ua = g.uL ? g.uL[u] : 0;
        const int64_t ub = g.uR ? g.uR[u] : 0;
        const T* a = arena + g.a_off + ua * g.a_key + scatter(m, g.apm, g.nam);
        const T* b = arena + g.b_off + ub * g.b_key + scatter(n, g.bpn, g.nbn);
        T acc = czero<T>();
        for (int64_t k = 0; k < g.K; ++k)
            acc = cfma(acc, a[scatter(k, g.apk, g.nak)], b[scatter(k, g.bpk, g.nbk)]);
        arena[g.c_off + u * g.c_key + m * g.N + n] = acc;
    }
}

// 64 x 64 output tile per CTA, 8-deep K slices, 256 threads with 4 x 4 each.
template <typename T>
__global__ void __launch_bounds__(256) k_gemm_tiled(const __grid_constant__ GemmDesc g, T* __restrict__ arena,
                                                    int64_t mt, int64_t nt) {
    __shared__ T As[8][64];
    __shared__ T Bs[8][64];
    __shared__ int64_t rowA[64], colB[64], kA[8], kB[8];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const bool a_along_k = g.nak > 0 && g.apk[0] == 0;
    const bool b_along_n = g.nbn > 0 && g.bpn[0] == 0;
    const int64_t n_tiles = g.kv * mt * nt;
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int64_t u = tile % g.kv;
        const int64_t rest = tile / g.kv;
        const int64_t m0 = (rest % mt) * 64;
        const int64_t n0 = (rest / mt) * 64;
        const int64_t ua = g.uL ? g.uL[u] : 0;
        const int64_t ub = g.uR ? g.uR[u] : 0;
        const T* A = arena + g.a_off + ua * g.a_key;
        const T* B = arena + g.b_off + ub * g.b_key;
        if (tid < 64) rowA[tid] = m0 + tid < g.M ? scatter(m0 + tid, g.apm, g.nam) : -1;
        else if (tid < 128) colB[tid - 64] = n0 + tid - 64 < g.N ? scatter(n0 + tid - 64, g.bpn, g.nbn) : -1;
        T acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = czero<T>();
        for (int64_t k0 = 0; k0 < g.K; k0 += 8) {
            if (tid < 8) kA[tid] = k0 + tid < g.K ? scatter(k0 + tid, g.apk, g.nak) : -1;
            else if (tid < 16) kB[tid - 8] = k0 + tid - 8 < g.K ? scatter(k0 + tid - 8, g.bpk, g.nbk) : -1;
            __syncthreads();
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const int e = tid + r * 256;
                int mm, kk;
                if (a_along_k) { kk = e & 7; mm = e >> 3; } else { mm = e & 63; kk = e >> 6; }
                As[kk][mm] = (rowA[mm] >= 0 && kA[kk] >= 0) ? A[rowA[mm] + kA[kk]] : czero<T>();
                int nn, kb;
                if (b_along_n) { nn = e & 63; kb = e >> 6; } else { kb = e & 7; nn = e >> 3; }
                Bs[kb][nn] = (colB[nn] >= 0 && kB[kb] >= 0) ? B[kB[kb] + colB[nn]] : czero<T>();
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) {
                T af[4], bf[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) af[i] = As[kk][ty * 4 + i];
#pragma unroll
                for (int j = 0; j < 4; ++j) bf[j] = Bs[kk][tx * 4 + j];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = cfma(acc[i][j], af[i], bf[j]);
            }
            __syncthreads();
        }
        T* C = arena + g.c_off + u * g.c_key;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int64_t m = m0 + ty * 4 + i;
            if (m >= g.M) continue;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int64_t n = n0 + tx * 4 + j;
                if (n < g.N) C[m * g.N + n] = acc[i][j];
            }
        }
        __syncthreads();
    }
}

// Keyed contractions with a deep summed index and a narrow result (for every
// key u a tile of at most 32 x 32 outputs over K >= 32 summed elements, e.g.
// the near-root nodes of sliced plans).  A CTA takes one (key, 32-row,
// 32-column) tile; every step stages a 64-deep chunk of A and B in shared
// memory (the next chunk is loaded into registers while this one is used),
// each of the 8 warps sums 8 of its columns of k into a full 32 x 32 partial
// tile (lane: 4 rows x 8 columns), and the warps' partial tiles are added in
// shared memory in three halving rounds before warp 0 writes the tile.
template <typename T>
__global__ void __launch_bounds__(256, 2) k_gemm_kdeep(const __grid_constant__ GemmDesc g, T* __restrict__ arena,
                                                       int64_t mt, int64_t nt) {
    extern __shared__ __align__(16) unsigned char kd_smem[];
    T* As = reinterpret_cast<T*>(kd_smem);                 // [kKdChunk][32]
    T* Bs = As + kKdChunk * kKdTile;                       // [kKdChunk][32]
    int64_t* rowA = reinterpret_cast<int64_t*>(Bs + kKdChunk * kKdTile);
    int64_t* colB = rowA + kKdTile;
    int64_t* kA = colB + kKdTile;                          // [2][kKdChunk] (double-buffered)
    int64_t* kB = kA + 2 * kKdChunk;
    T* red = As;                                           // [4][32 * 32] after the last chunk
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int rg = lane >> 2, cg = lane & 3;               // rows 4 rg .. 4 rg + 3, columns 8 cg .. 8 cg + 7
    const bool a_along_k = g.nak > 0 && g.apk[0] == 0;
    const bool b_along_n = g.nbn > 0 && g.bpn[0] == 0;
    const int64_t n_tiles = g.kv * mt * nt;
    const int64_t n_chunks = (g.K + kKdChunk - 1) / kKdChunk;
    constexpr int kPer = kKdChunk * kKdTile / 256;         // staged elements per thread per operand
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int64_t u = tile % g.kv;
        const int64_t rest = tile / g.kv;
        const int64_t m0 = (rest % mt) * kKdTile;
        const int64_t n0 = (rest / mt) * kKdTile;
        const T* A = arena + g.a_off + (g.uL ? int64_t(g.uL[u]) : 0) * g.a_key;
        const T* B = arena + g.b_off + (g.uR ? int64_t(g.uR[u]) : 0) * g.b_key;
        if (tid < kKdTile) rowA[tid] = m0 + tid < g.M ? scatter(m0 + tid, g.apm, g.nam) : -1;
        else if (tid < 2 * kKdTile) colB[tid - kKdTile] = n0 + tid - kKdTile < g.N ? scatter(n0 + tid - kKdTile, g.bpn, g.nbn) : -1;
        auto k_offsets = [&](int64_t c, int buf) {
            if (tid < kKdChunk) {
                const int64_t k = c * kKdChunk + tid;
                kA[buf * kKdChunk + tid] = k < g.K ? scatter(k, g.apk, g.nak) : -1;
            } else if (tid < 2 * kKdChunk) {
                const int64_t k = c * kKdChunk + tid - kKdChunk;
                kB[buf * kKdChunk + tid - kKdChunk] = k < g.K ? scatter(k, g.bpk, g.nbk) : -1;
            }
        };
        // element e of a chunk: (row or column index, k) with the operand's
        // lowest address dimension fastest across threads
        auto a_idx = [&](int e, int& mm, int& kk) {
            if (a_along_k) { kk = e % kKdChunk; mm = e / kKdChunk; } else { mm = e % kKdTile; kk = e / kKdTile; }
        };
        auto b_idx = [&](int e, int& nn, int& kk) {
            if (b_along_n) { nn = e % kKdTile; kk = e / kKdTile; } else { kk = e % kKdChunk; nn = e / kKdChunk; }
        };
        T ra[kPer], rb[kPer];
        auto load = [&](int buf) {
#pragma unroll
            for (int j = 0; j < kPer; ++j) {
                int mm, kk, nn, kb;
                a_idx(tid + j * 256, mm, kk);
                const int64_t ka = kA[buf * kKdChunk + kk];
                ra[j] = (rowA[mm] >= 0 && ka >= 0) ? A[rowA[mm] + ka] : czero<T>();
                b_idx(tid + j * 256, nn, kb);
                const int64_t kbo = kB[buf * kKdChunk + kb];
                rb[j] = (colB[nn] >= 0 && kbo >= 0) ? B[kbo + colB[nn]] : czero<T>();
            }
        };
        k_offsets(0, 0);
        __syncthreads();
        load(0);
        T acc[4][8];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = czero<T>();
        for (int64_t c = 0; c < n_chunks; ++c) {
            const int buf = int(c & 1);
#pragma unroll
            for (int j = 0; j < kPer; ++j) {
                int mm, kk, nn, kb;
                a_idx(tid + j * 256, mm, kk);
                As[kk * kKdTile + mm] = ra[j];
                b_idx(tid + j * 256, nn, kb);
                Bs[kb * kKdTile + nn] = rb[j];
            }
            if (c + 1 < n_chunks) k_offsets(c + 1, buf ^ 1);
            __syncthreads();
            if (c + 1 < n_chunks) load(buf ^ 1);   // next chunk in flight during the sums
#pragma unroll
            for (int kk = warp * (kKdChunk / 8); kk < (warp + 1) * (kKdChunk / 8); ++kk) {
                T af[4], bf[8];
#pragma unroll
                for (int i = 0; i < 4; ++i) af[i] = As[kk * kKdTile + rg * 4 + i];
#pragma unroll
                for (int j = 0; j < 8; ++j) bf[j] = Bs[kk * kKdTile + cg * 8 + j];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[i][j] = cfma(acc[i][j], af[i], bf[j]);
            }
            __syncthreads();
        }
        // sum the 8 warps' partial tiles: 8 -> 4 -> 2 -> 1
#pragma unroll
        for (int half = 4; half >= 1; half >>= 1) {
            if (warp >= half && warp < 2 * half) {
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) red[(warp - half) * 1024 + (rg * 4 + i) * 32 + cg * 8 + j] = acc[i][j];
            }
            __syncthreads();
            if (warp < half) {
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[i][j] = cadd(acc[i][j], red[warp * 1024 + (rg * 4 + i) * 32 + cg * 8 + j]);
            }
            __syncthreads();
        }
        if (warp == 0) {
            T* C = arena + g.c_off + u * g.c_key;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int64_t m = m0 + rg * 4 + i;
                if (m >= g.M) continue;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int64_t n = n0 + cg * 8 + j;
                    if (n < g.N) C[m * g.N + n] = acc[i][j];
                }
            }
        }
        __syncthreads();
    }
}

template <typename T>
constexpr size_t kdeep_smem_bytes() {
    return size_t(2 * kKdChunk * kKdTile) * sizeof(T) + size_t(2 * kKdTile + 4 * kKdChunk) * sizeof(int64_t);
}

// N == 1: one thread per (left-key group, row m); the A row is shared by all
// keys of the group (keys are sorted by their left key, so groups are runs).
constexpr int kGemvK = 256;
template <typename T>
__global__ void k_gemm_gemv(const __grid_constant__ GemmDesc g, T* __restrict__ arena) {
    __shared__ int64_t kA[kGemvK], kB[kGemvK];
    const bool table = g.K <= kGemvK;
    if (table)
        for (int k = threadIdx.x; k < g.K; k += blockDim.x) {
            kA[k] = scatter(k, g.apk, g.nak);
            kB[k] = scatter(k, g.bpk, g.nbk);
        }
    __syncthreads();
    const int64_t total = g.n_groups * g.M;
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total;
         e += int64_t(gridDim.x) * blockDim.x) {
        const int64_t m = e % g.M;
        const int64_t grp = e / g.M;
        const int64_t u0 = g.gstart ? g.gstart[grp] : 0;
        const int64_t u1 = g.gstart ? g.gstart[grp + 1] : g.kv;
        if (u1 <= u0) continue;
        const int64_t ua = g.uL ? g.uL[u0] : 0;
        const T* a = arena + g.a_off + ua * g.a_key + scatter(m, g.apm, g.nam);
        for (int64_t u = u0; u < u1; ++u) {
            const int64_t ub = g.uR ? g.uR[u] : 0;
            const T* b = arena + g.b_off + ub * g.b_key;
            T acc = czero<T>();
            if (table) {
                for (int64_t k = 0; k < g.K; ++k) acc = cfma(acc, a[kA[k]], b[kB[k]]);
            } else {
                for (int64_t k = 0; k < g.K; ++k)
                    acc = cfma(acc, a[scatter(k, g.apk, g.nak)], b[scatter(k, g.bpk, g.nbk)]);
            }
            arena[g.c_off + u * g.c_key + m] = acc;
        }
    }
}

// M == N == 1: a warp per key, lanes split K, shuffle reduction.
template <typename T>
__global__ void k_gemm_tail(const __grid_constant__ GemmDesc g, T* __restrict__ arena) {
    // one warp per output (key u, row m) of an N = 1 contraction: lanes
    // stride the summed index, a shuffle tree adds their partial sums
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    const int64_t total = g.kv * g.M;
    for (int64_t w = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5; w < total; w += warps) {
        const int64_t u = w / g.M, m = w - u * g.M;
        const int64_t ua = g.uL ? g.uL[u] : 0;
        const int64_t ub = g.uR ? g.uR[u] : 0;
        const T* a = arena + g.a_off + ua * g.a_key + scatter(m, g.apm, g.nam);
        const T* b = arena + g.b_off + ub * g.b_key;
        T acc = czero<T>();
        for (int64_t k = lane; k < g.K; k += 32)
            acc = cfma(acc, a[scatter(k, g.apk, g.nak)], b[scatter(k, g.bpk, g.nbk)]);
        for (int d = 16; d > 0; d >>= 1) acc = cadd(acc, shfl_down(acc, d));
        if (lane == 0) arena[g.c_off + u * g.c_key + m] = acc;
    }
}

template <typename T>
cudaError_t launch_gemm(int kernel, const GemmDesc& g, T* arena, cudaStream_t st) {
    const int cap = 152 * 32;
    switch (kernel) {
        case GK_TILED: {
            const int64_t mt = (g.M + 63) / 64, nt = (g.N + 63) / 64;
            k_gemm_tiled<T><<<grid_for(g.kv * mt * nt, 1, cap), 256, 0, st>>>(g, arena, mt, nt);
            break;
        }
        case GK_GEMV:
            k_gemm_gemv<T><<<grid_for(g.n_groups * g.M, 256, cap), 256, 0, st>>>(g, arena);
            break;
        case GK_KDEEP: {
            const int64_t mt = (g.M + kKdTile - 1) / kKdTile, nt = (g.N + kKdTile - 1) / kKdTile;
            k_gemm_kdeep<T><<<grid_for(g.kv * mt * nt, 1, 152 * 2), 256, kdeep_smem_bytes<T>(), st>>>(g, arena, mt, nt);
            break;
        }
        case GK_TAIL:
            k_gemm_tail<T><<<grid_for(g.kv * g.M * 32, 256, cap), 256, 0, st>>>(g, arena);
            break;
        default:
            k_gemm_generic<T><<<grid_for(g.kv * g.M * g.N, 256, cap), 256, 0, st>>>(g, arena);
    }
    return cudaGetLastError();
}

// Memory-bound contraction (M large, K and N <= 64): a CTA loads R rows x all
// K of A as contiguous address runs, transposes them in shared memory, then
// every key of the left-key group multiplies the tile by its B and writes R x N
// contiguous outputs.  Each thread owns one row and NPT consecutive columns.
// The tile geometry is the same for every tile, so each thread computes the
// address offsets and shared-memory slots of its EPT tile elements once.
template <int NPT>
__device__ __forceinline__ void load_vec(const float2* p, float2* out) {
    if constexpr (NPT % 2 == 0) {
#pragma unroll
        for (int j = 0; j < NPT; j += 2) {
            const float4 q = *reinterpret_cast<const float4*>(p + j);
            out[j] = make_float2(q.x, q.y);
            out[j + 1] = make_float2(q.z, q.w);
        }
    } else {
#pragma unroll
        for (int j = 0; j < NPT; ++j) out[j] = p[j];
    }
}
template <int NPT>
__device__ __forceinline__ void load_vec(const double2* p, double2* out) {
#pragma unroll
    for (int j = 0; j < NPT; ++j) out[j] = p[j];
}
template <int NPT>
__device__ __forceinline__ void store_vec(float2* p, const float2* v) {
    if constexpr (NPT % 2 == 0) {
#pragma unroll
        for (int j = 0; j < NPT; j += 2)
            *reinterpret_cast<float4*>(p + j) = make_float4(v[j].x, v[j].y, v[j + 1].x, v[j + 1].y);
    } else {
#pragma unroll
        for (int j = 0; j < NPT; ++j) p[j] = v[j];
    }
}
template <int NPT>
__device__ __forceinline__ void store_vec(double2* p, const double2* v) {
#pragma unroll
    for (int j = 0; j < NPT; ++j) p[j] = v[j];
}

__device__ __forceinline__ void cp_async_el(float2* smem, const float2* gmem) {
    const unsigned sa = unsigned(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_el(double2* smem, const double2* gmem) {
    const unsigned sa = unsigned(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <typename T, int NPT>
__global__ void __launch_bounds__(256, 2) k_gemm_stream(const __grid_constant__ GemmDesc g,
                                                        const __grid_constant__ StreamDesc s,
                                                        T* __restrict__ arena) {
    extern __shared__ __align__(16) unsigned char sm_stream[];
    const int R = s.R, K = int(g.K), N = int(g.N);
    const int ldA = R + 1, ldB = N + (NPT > 1 ? 2 : 1);
    const int a_sz = (K * ldA + 1) & ~1;
    T* bufs = reinterpret_cast<T*>(sm_stream);  // kStreamStages A tiles [K][R+1], then B [K][ldB]
    T* Bs = bufs + kStreamStages * a_sz;
    const int tid = threadIdx.x;
    const int tile_elems = R * K;
    int32_t off[kStreamEPT];
    int slot[kStreamEPT];
#pragma unroll
    for (int j = 0; j < kStreamEPT; ++j) {
        const int e = tid + j * 256;
        off[j] = 0;
        slot[j] = -1;
        if (e < tile_elems) {
            int r = 0, k = 0, ri = 0, ki = 0;
            int32_t o = 0;
            for (int i = 0; i < s.T; ++i) {
                const int bit = (e >> i) & 1;
                if ((s.is_k >> i) & 1) k |= bit << ki++;
                else r |= bit << ri++;
                if (bit) o |= int32_t(1) << s.pos[i];
            }
            off[j] = o;
            slot[j] = k * ldA + r;
        }
    }
    const int TPR = N >= NPT ? N / NPT : 1;
    const int RG = 256 / TPR;
    const int my_rg = tid / TPR, my_c = tid % TPR;
    const int64_t tiles_per_group = (g.M + R - 1) / R;
    const int64_t n_tiles = g.n_groups * tiles_per_group;
    const bool single = g.n_groups == 1 && g.kv == 1;
    auto load_B = [&](int64_t u) {
        const int64_t ub = g.uR ? g.uR[u] : 0;
        const T* B = arena + g.b_off + ub * g.b_key;
        for (int e = tid; e < K * N; e += 256) {
            const int k = e / N, n = e % N;
            Bs[k * ldB + n] = B[scatter(k, g.bpk, g.nbk) + scatter(n, g.bpn, g.nbn)];
        }
    };
    auto issue = [&](int64_t tile, T* buf) {
        const int64_t grp = tile / tiles_per_group;
        const int64_t mt = tile % tiles_per_group;
        const int64_t u0 = g.gstart ? g.gstart[grp] : 0;
        const int64_t ua = g.uL ? g.uL[u0] : 0;
        const T* A = arena + g.a_off + ua * g.a_key + scatter(mt * R, g.apm, g.nam);
        const int64_t rows_left = g.M - mt * R;
#pragma unroll
        for (int j = 0; j < kStreamEPT; ++j) {
            if (slot[j] < 0) continue;
            if (rows_left >= R || (slot[j] % ldA) < rows_left) cp_async_el(buf + slot[j], A + off[j]);
            else buf[slot[j]] = czero<T>();
        }
    };
    if (single) load_B(0);
    // ring of kStreamStages tiles: the loads of the next kStreamStages-1
    // tiles are in flight while one tile is multiplied
#pragma unroll
    for (int p = 0; p < kStreamStages - 1; ++p) {
        const int64_t tl = blockIdx.x + int64_t(p) * gridDim.x;
        if (tl < n_tiles) issue(tl, bufs + p * a_sz);
        cp_async_commit();
    }
    int64_t tile = blockIdx.x;
    for (int it = 0; tile < n_tiles; tile += gridDim.x, ++it) {
        T* cur = bufs + (it % kStreamStages) * a_sz;
        const int64_t ahead = tile + int64_t(kStreamStages - 1) * gridDim.x;
        if (ahead < n_tiles) issue(ahead, bufs + ((it + kStreamStages - 1) % kStreamStages) * a_sz);
        cp_async_commit();
        cp_async_wait<kStreamStages - 1>();
        __syncthreads();
        const int64_t grp = tile / tiles_per_group;
        const int64_t mt = tile % tiles_per_group;
        const int64_t u0 = g.gstart ? g.gstart[grp] : 0;
        const int64_t u1 = g.gstart ? g.gstart[grp + 1] : g.kv;
        const int64_t rows_left = g.M - mt * R;
        if (N == 1 && !single) {
            // memo-trie levels: many keys share this A tile; stage the B
            // vectors of a batch of keys at once, then one (row, key) dot
            // product per thread slot
            const int kb_max = kStreamBKeys / K;
            for (int64_t ub0 = u0; ub0 < u1; ub0 += kb_max) {
                const int64_t left_keys = u1 - ub0;
                const int nb = left_keys < kb_max ? int(left_keys) : kb_max;
                for (int e = tid; e < nb * K; e += 256) {
                    const int j = e / K, k = e % K;
                    const int64_t ub = g.uR ? g.uR[ub0 + j] : 0;
                    Bs[e] = arena[g.b_off + ub * g.b_key + scatter(k, g.bpk, g.nbk)];
                }
                __syncthreads();
                const int rows = rows_left < R ? int(rows_left) : R;
                if (K <= 16) {
                    // a thread keeps its row of A in registers and walks its
                    // share of the keys; a warp covers 32 consecutive rows of
                    // one key, so B is read as a broadcast and C stores coalesce
                    const int S = R >= 256 ? 1 : 256 / R;   // threads per row
                    const int rs = R >= 256 ? 256 : R;       // row stride
                    for (int r = R >= 256 ? tid : tid % R; r < rows; r += rs) {
                        T a[16];
#pragma unroll
                        for (int k = 0; k < 16; ++k) a[k] = k < K ? cur[k * ldA + r] : czero<T>();
                        for (int j = R >= 256 ? 0 : tid / R; j < nb; j += S) {
                            const T* b = Bs + j * K;
                            T acc = czero<T>();
#pragma unroll
                            for (int k = 0; k < 16; ++k)
                                if (k < K) acc = cfma(acc, a[k], b[k]);
                            arena[g.c_off + (ub0 + j) * g.c_key + mt * R + r] = acc;
                        }
                    }
                } else {
                    for (int pr = tid; pr < rows * nb; pr += 256) {
                        const int r = pr % rows, j = pr / rows;
                        T acc = czero<T>();
                        for (int k = 0; k < K; ++k) acc = cfma(acc, cur[k * ldA + r], Bs[j * K + k]);
                        arena[g.c_off + (ub0 + j) * g.c_key + mt * R + r] = acc;
                    }
                }
                __syncthreads();
            }
            continue;
        }
        for (int64_t u = u0; u < u1; ++u) {
            if (!single) {
                load_B(u);
                __syncthreads();
            }
            if (my_c * NPT < N) {
                for (int r = my_rg; r < R && r < rows_left; r += RG) {
                    T acc[NPT];
#pragma unroll
                    for (int j = 0; j < NPT; ++j) acc[j] = czero<T>();
                    for (int k = 0; k < K; ++k) {
                        const T a = cur[k * ldA + r];
                        T b[NPT];
                        load_vec<NPT>(Bs + k * ldB + my_c * NPT, b);
#pragma unroll
                        for (int j = 0; j < NPT; ++j) acc[j] = cfma(acc[j], a, b[j]);
                    }
                    store_vec<NPT>(arena + g.c_off + u * g.c_key + (mt * R + r) * N + my_c * NPT, acc);
                }
            }
            if (!single) __syncthreads();
        }
        __syncthreads();
    }
    cp_async_wait<0>();
}

// ---- memo-trie levels: many keys per A tile, N = 1 ---------------------------------
// C_u[m] = sum_k A_{uL(u)}[m][k] B_{uR(u)}[k] for the keys u of each left-key
// group.  A prep kernel writes every group's A offset and packs every key's B
// vector contiguously (keys are ordered by uL then uR, so a group's vectors
// are one run); the main loop then loads a tile's A rows and its group's B
// vectors together with cp.async, kStreamStages - 1 tiles ahead, and reads
// the next tile's group data one iteration before it issues those loads, so
// no dependent global read sits on the critical path.
template <typename T>
__global__ void k_memo_prep(const __grid_constant__ GemmDesc g, const T* __restrict__ arena, int64_t* grp_a,
                            T* bpack) {
    const int64_t K = g.K;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < g.n_groups; i += stride)
        grp_a[i] = int64_t(g.uL[g.gstart[i]]) * g.a_key;
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < g.kv * K; e += stride) {
        const int64_t u = e / K, k = e % K;
        bpack[e] = arena[g.b_off + int64_t(g.uR[u]) * g.b_key + scatter(k, g.bpk, g.nbk)];
    }
}

// Rows x keys of one memo-level tile with K = 16 (complex64): thread tid
// takes row tid % R (R < 256: 256 / R threads share a row and take every
// (256 / R)-th key) and keeps the row's 16 values in registers; the keys'
// B vectors (16 values each, 16-byte aligned) are read two values at a time.
// C points at (first key of the batch, first row of the tile); key j's row r
// is C[j * c_key + r].
__device__ __forceinline__ void memo_rows_k16(const float2* __restrict__ cur, int ldA, const float2* __restrict__ Bv,
                                              float2* __restrict__ C, int64_t c_key, int R, int rows, int nb) {
    const int tid = threadIdx.x;
    const int S = R >= 256 ? 1 : 256 / R;
    const int rs = R >= 256 ? 256 : R;
    const int j0 = R >= 256 ? 0 : tid / R;
    for (int r = R >= 256 ? tid : tid % R; r < rows; r += rs) {
        float2 a[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) a[k] = cur[k * ldA + r];
        int j = j0;
        for (; j + S < nb; j += 2 * S) {
            const float4* b0 = reinterpret_cast<const float4*>(Bv + j * 16);
            const float4* b1 = reinterpret_cast<const float4*>(Bv + (j + S) * 16);
            float2 c0 = make_float2(0.f, 0.f), c1 = make_float2(0.f, 0.f);
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) {
                const float4 q0 = b0[kk], q1 = b1[kk];
                c0 = cfma(c0, a[2 * kk], make_float2(q0.x, q0.y));
                c0 = cfma(c0, a[2 * kk + 1], make_float2(q0.z, q0.w));
                c1 = cfma(c1, a[2 * kk], make_float2(q1.x, q1.y));
                c1 = cfma(c1, a[2 * kk + 1], make_float2(q1.z, q1.w));
            }
            C[j * c_key + r] = c0;
            C[(j + S) * c_key + r] = c1;
        }
        if (j < nb) {
            const float4* b0 = reinterpret_cast<const float4*>(Bv + j * 16);
            float2 c0 = make_float2(0.f, 0.f);
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) {
                const float4 q0 = b0[kk];
                c0 = cfma(c0, a[2 * kk], make_float2(q0.x, q0.y));
                c0 = cfma(c0, a[2 * kk + 1], make_float2(q0.z, q0.w));
            }
            C[j * c_key + r] = c0;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(256, 2) k_gemm_memo(const __grid_constant__ GemmDesc g,
                                                      const __grid_constant__ StreamDesc s, T* __restrict__ arena,
                                                      const int64_t* __restrict__ grp_a,
                                                      const T* __restrict__ bpack) {
    extern __shared__ __align__(16) unsigned char sm_memo[];
    const int R = s.R, K = int(g.K);
    const int ldA = R + 1;
    const int a_sz = (K * ldA + 1) & ~1;
    T* abuf = reinterpret_cast<T*>(sm_memo);                 // kStreamStages x [K][R+1]
    T* bbuf = abuf + kStreamStages * a_sz;                     // kStreamStages x kMemoBPre
    T* Bs = bbuf + kStreamStages * kMemoBPre;                  // synchronous staging (large groups)
    int64_t* rowoff = reinterpret_cast<int64_t*>(Bs + kStreamBKeys);  // per row bit above the tile
    int64_t* meta = rowoff + kMaxLegs;                         // per stage: u0, u1
    const int tid = threadIdx.x;
    for (int i = tid; i < g.nam; i += 256) rowoff[i] = int64_t(1) << g.apm[i];
    const int tile_elems = R * K;
    int32_t off[kStreamEPT];
    int slot[kStreamEPT];
#pragma unroll
    for (int j = 0; j < kStreamEPT; ++j) {
        const int e = tid + j * 256;
        off[j] = 0;
        slot[j] = -1;
        if (e < tile_elems) {
            int r = 0, k = 0, ri = 0, ki = 0;
            int32_t o = 0;
            for (int i = 0; i < s.T; ++i) {
                const int bit = (e >> i) & 1;
                if ((s.is_k >> i) & 1) k |= bit << ki++;
                else r |= bit << ri++;
                if (bit) o |= int32_t(1) << s.pos[i];
            }
            off[j] = o;
            slot[j] = k * ldA + r;
        }
    }
    __syncthreads();
    const int64_t tpg = (g.M + R - 1) / R;   // tiles per group
    const int64_t n_tiles = g.n_groups * tpg;
    struct Meta {
        int64_t u0, u1, aoff;
    };
    auto load_meta = [&](int64_t tile) {
        Meta m{0, 0, 0};
        if (tile < n_tiles) {
            const int64_t grp = tile / tpg;
            m.u0 = g.gstart[grp];
            m.u1 = g.gstart[grp + 1];
            m.aoff = grp_a[grp];
        }
        return m;
    };
    auto issue = [&](int64_t tile, int stage, const Meta& m) {
        const int64_t mt = tile % tpg;
        int64_t ro = 0;
        for (int64_t x = (mt * R) >> s.tm, i = s.tm; x != 0; x >>= 1, ++i)
            if (x & 1) ro += rowoff[i];
        const T* A = arena + g.a_off + m.aoff + ro;
        const int64_t rows_left = g.M - mt * R;
        T* buf = abuf + stage * a_sz;
#pragma unroll
        for (int j = 0; j < kStreamEPT; ++j) {
            if (slot[j] < 0) continue;
            if (rows_left >= R || (slot[j] % ldA) < rows_left) cp_async_el(buf + slot[j], A + off[j]);
            else buf[slot[j]] = czero<T>();
        }
        const int64_t nbk = (m.u1 - m.u0) * K;
        if (nbk <= kMemoBPre) {
            T* bb = bbuf + stage * kMemoBPre;
            for (int64_t e = tid; e < nbk; e += 256) cp_async_el(bb + e, bpack + m.u0 * K + e);
        }
        if (tid == 0) {
            meta[2 * stage] = m.u0;
            meta[2 * stage + 1] = m.u1;
        }
    };
    const int64_t G = gridDim.x;
#pragma unroll
    for (int p = 0; p < kStreamStages - 1; ++p) {
        const int64_t tl = blockIdx.x + int64_t(p) * G;
        if (tl < n_tiles) issue(tl, p, load_meta(tl));
        cp_async_commit();
    }
    Meta next = load_meta(blockIdx.x + int64_t(kStreamStages - 1) * G);
    int64_t tile = blockIdx.x;
    for (int it = 0; tile < n_tiles; tile += G, ++it) {
        const int stage = it % kStreamStages;
        const int64_t ahead = tile + int64_t(kStreamStages - 1) * G;
        const Meta m = next;
        next = load_meta(ahead + G);   // used by the next iteration
        if (ahead < n_tiles) issue(ahead, (it + kStreamStages - 1) % kStreamStages, m);
        cp_async_commit();
        cp_async_wait<kStreamStages - 1>();
        __syncthreads();
        const T* cur = abuf + stage * a_sz;
        const int64_t u0 = meta[2 * stage], u1 = meta[2 * stage + 1];
        const int64_t mt = tile % tpg;
        const int64_t rows_left = g.M - mt * R;
        const int rows = rows_left < R ? int(rows_left) : R;
        const int64_t nkeys = u1 - u0;
        const bool pre = nkeys * K <= kMemoBPre;
        const int kb_max = pre ? int(nkeys) : kStreamBKeys / K;
        for (int64_t ub0 = u0; ub0 < u1; ub0 += kb_max) {
            const int nb = u1 - ub0 < kb_max ? int(u1 - ub0) : kb_max;
            const T* Bv = bbuf + stage * kMemoBPre;
            if (!pre) {
                for (int e = tid; e < nb * K; e += 256) Bs[e] = bpack[ub0 * K + e];
                __syncthreads();
                Bv = Bs;
            }
            if (sizeof(T) == 8 && K == 16) {
                // the memo-trie levels of grid plans: 16 summed values (four
                // output bits), complex64.  Compile-time K, B read as float4,
                // two keys per pass over the row's values in registers
                memo_rows_k16(reinterpret_cast<const float2*>(cur), ldA, reinterpret_cast<const float2*>(Bv),
                              reinterpret_cast<float2*>(arena) + g.c_off + ub0 * g.c_key + mt * R, g.c_key,
                              R, rows, nb);
            } else if (K <= 16) {
                const int S = R >= 256 ? 1 : 256 / R;   // threads per row
                const int rs = R >= 256 ? 256 : R;
                for (int r = R >= 256 ? tid : tid % R; r < rows; r += rs) {
                    T a[16];
#pragma unroll
                    for (int k = 0; k < 16; ++k) a[k] = k < K ? cur[k * ldA + r] : czero<T>();
                    for (int j = R >= 256 ? 0 : tid / R; j < nb; j += S) {
                        const T* b = Bv + j * K;
                        T acc = czero<T>();
#pragma unroll
                        for (int k = 0; k < 16; ++k)
                            if (k < K) acc = cfma(acc, a[k], b[k]);
                        arena[g.c_off + (ub0 + j) * g.c_key + mt * R + r] = acc;
                    }
                }
            } else {
                for (int pr = tid; pr < rows * nb; pr += 256) {
                    const int r = pr % rows, j = pr / rows;
                    T acc = czero<T>();
                    for (int k = 0; k < K; ++k) acc = cfma(acc, cur[k * ldA + r], Bv[j * K + k]);
                    arena[g.c_off + (ub0 + j) * g.c_key + mt * R + r] = acc;
                }
            }
            if (!pre) __syncthreads();
        }
        __syncthreads();
    }
    cp_async_wait<0>();
}

template <typename T>
cudaError_t launch_memo_prep(const GemmDesc& g, T* arena, char* scratch, cudaStream_t st) {
    int64_t* grp_a = reinterpret_cast<int64_t*>(scratch);
    T* bpack = reinterpret_cast<T*>(scratch + ((size_t(g.n_groups) * 8 + 255) & ~size_t(255)));
    k_memo_prep<T><<<grid_for(g.kv * g.K, 256, 152 * 8), 256, 0, st>>>(g, arena, grp_a, bpack);
    return cudaGetLastError();
}
template cudaError_t launch_memo_prep<float2>(const GemmDesc&, float2*, char*, cudaStream_t);

size_t memo_scratch_bytes(int64_t n_groups, int64_t kv, int64_t K, size_t elem) {
    return size_t(n_groups) * 8 + 256 + size_t(kv * K) * elem;
}

template <typename T>
cudaError_t launch_gemm_memo(const GemmDesc& g, const StreamDesc& s, T* arena, char* scratch, cudaStream_t st) {
    int64_t* grp_a = reinterpret_cast<int64_t*>(scratch);
    T* bpack = reinterpret_cast<T*>(scratch + ((size_t(g.n_groups) * 8 + 255) & ~size_t(255)));
    k_memo_prep<T><<<grid_for(g.kv * g.K, 256, 152 * 8), 256, 0, st>>>(g, arena, grp_a, bpack);
    const size_t a_sz = (size_t(g.K) * (s.R + 1) + 1) & ~size_t(1);
    const size_t smem = sizeof(T) * (kStreamStages * (a_sz + kMemoBPre) + kStreamBKeys) + 8 * (kMaxLegs + 2 * kStreamStages);
    const int64_t tiles = g.n_groups * ((g.M + s.R - 1) / s.R);
    k_gemm_memo<T><<<grid_for(tiles, 1, 152 * 8), 256, smem, st>>>(g, s, arena, grp_a, bpack);
    return cudaGetLastError();
}

// ---- outer products: K = 1, one key, natural layouts ------------------------------
// C[m][n] = A[m] B[n] (the summed index is empty): all of the work is writing
// C.  Thread t owns the column pair p = t mod (N / 2) on every row it visits,
// keeps B[2p] and B[2p + 1] in registers and writes the two results of a row
// as one vector store, so a warp writes whole rows (512 contiguous bytes for
// N = 64 complex64); the lanes of a row read its A value as one broadcast.
// Four rows per thread are loaded before any is stored.
template <typename T>
__global__ void __launch_bounds__(256) k_outer(const __grid_constant__ GemmDesc g, T* __restrict__ arena) {
    const int P = int(g.N >> 1);   // column pairs per row, a power of two dividing 256
    const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int p = int(tid & (P - 1));
    const int64_t ua = g.uL ? g.uL[0] : 0, ub = g.uR ? g.uR[0] : 0;
    const T* __restrict__ A = arena + g.a_off + ua * g.a_key;
    const T* __restrict__ B = arena + g.b_off + ub * g.b_key;
    T* __restrict__ C = arena + g.c_off;
    const T b0 = B[2 * p], b1 = B[2 * p + 1];
    const int64_t rs = int64_t(gridDim.x) * blockDim.x / P;   // rows per pass of the grid
    constexpr int U = 4;
    for (int64_t r0 = tid / P; r0 < g.M; r0 += U * rs) {
        T a[U];
#pragma unroll
        for (int u = 0; u < U; ++u) a[u] = r0 + u * rs < g.M ? A[r0 + u * rs] : czero<T>();
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t r = r0 + u * rs;
            if (r < g.M) {
                const T v[2] = {cfma(czero<T>(), a[u], b0), cfma(czero<T>(), a[u], b1)};
                store_vec<2>(C + r * g.N + 2 * p, v);
            }
        }
    }
}

// the outer-product kernel applies: K = 1, one key, A's rows and B's columns
// at consecutive addresses from bit 0, C row-major, N = 2 .. 512 a power of
// two, and 16-byte aligned result pairs and B pairs
template <typename T>
bool outer_fits(const GemmDesc& g) {
    if (g.K != 1 || g.kv != 1 || g.n_groups != 1 || !g.c_natural || g.nak != 0 || g.nbk != 0) return false;
    if (g.N < 2 || g.N > 512 || (g.N & (g.N - 1)) != 0 || g.M != (int64_t(1) << g.nam) || g.N != (int64_t(1) << g.nbn))
        return false;
    for (int i = 0; i < g.nam; ++i)
        if (g.apm[i] != i) return false;
    for (int i = 0; i < g.nbn; ++i)
        if (g.bpn[i] != i) return false;
    return sizeof(T) == 16 || (g.c_off % 2 == 0 && g.b_off % 2 == 0 && g.b_key % 2 == 0);
}

template <typename T>
cudaError_t launch_gemm_stream(const GemmDesc& g, const StreamDesc& s, T* arena, cudaStream_t st) {
    if (outer_fits<T>(g)) {
        k_outer<T><<<152 * 8, 256, 0, st>>>(g, arena);
        return cudaGetLastError();
    }
    const size_t a_sz = (size_t(g.K) * (s.R + 1) + 1) & ~size_t(1);
    const size_t b_sz = g.N == 1 ? size_t(kStreamBKeys) : size_t(g.K) * (g.N + 2);
    const size_t smem = sizeof(T) * (kStreamStages * a_sz + b_sz);
    const int64_t tiles = g.n_groups * ((g.M + s.R - 1) / s.R);
    const int grid = grid_for(tiles, 1, 152 * 8);
    switch (s.npt) {
#define XEB_STREAM_CASE(P)                                    \
    case P:                                                   \
        k_gemm_stream<T, P><<<grid, 256, smem, st>>>(g, s, arena); \
        break;
        XEB_STREAM_CASE(1)
        XEB_STREAM_CASE(2)
        XEB_STREAM_CASE(4)
        XEB_STREAM_CASE(8)
        XEB_STREAM_CASE(16)
#undef XEB_STREAM_CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ---- a6/a7 -------------------------------------------------------------------------

__device__ __forceinline__ double2 to_d2(float2 v) { return make_double2(v.x, v.y); }
__device__ __forceinline__ double2 to_d2(double2 v) { return v; }

template <typename T>
__global__ void k_root_accum(const T* root, double2* acc, int64_t kv) {
    for (int64_t u = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; u < kv; u += int64_t(gridDim.x) * blockDim.x) {
        const double2 r = to_d2(root[u]);
        double2 a = acc[u];
        a.x += r.x;
        a.y += r.y;
        acc[u] = a;
    }
}

template <typename T>
cudaError_t launch_root_accum(const T* root, double2* acc, int64_t kv, cudaStream_t st) {
    k_root_accum<T><<<grid_for(kv, 256, 1024), 256, 0, st>>>(root, acc, kv);
    return cudaGetLastError();
}

// amps[i * 2^w + x] = the root value of bitstring i's key at open-qubit
// value x; block partial sums of p and p^2 over all k 2^w values.
__global__ void __launch_bounds__(256) k_gather_xeb(const double2* acc, const int32_t* key_root, int64_t k,
                                                    const RootMap rm, double2* amps, double* partials) {
    __shared__ double s1[256], s2[256];
    double a1 = 0.0, a2 = 0.0;
    const int64_t total = k << rm.w;
    const int64_t xmask = (int64_t(1) << rm.w) - 1;
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
        const int64_t x = e & xmask;
        int64_t off = 0;
        for (int j = 0; j < rm.w; ++j)
            if ((x >> j) & 1) off |= int64_t(1) << rm.pos[j];
        const double2 a = acc[(int64_t(key_root[e >> rm.w]) << rm.w) + off];
        amps[e] = a;
        const double p = a.x * a.x + a.y * a.y;
        a1 += p;
        a2 += p * p;
    }
    s1[threadIdx.x] = a1;
    s2[threadIdx.x] = a2;
    __syncthreads();
    for (int d = 128; d > 0; d >>= 1) {
        if (threadIdx.x < d) {
            s1[threadIdx.x] += s1[threadIdx.x + d];
            s2[threadIdx.x] += s2[threadIdx.x + d];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = s1[0];
        partials[2 * blockIdx.x + 1] = s2[0];
    }
}

__global__ void __launch_bounds__(256) k_xeb_final(const double* partials, int nb, int64_t k, int n,
                                                   double* result) {
    __shared__ double s1[256], s2[256];
    double a1 = 0.0, a2 = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        a1 += partials[2 * b];
        a2 += partials[2 * b + 1];
    }
    s1[threadIdx.x] = a1;
    s2[threadIdx.x] = a2;
    __syncthreads();
    for (int d = 128; d > 0; d >>= 1) {
        if (threadIdx.x < d) {
            s1[threadIdx.x] += s1[threadIdx.x + d];
            s2[threadIdx.x] += s2[threadIdx.x + d];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double scale = ldexp(1.0, n);
        const double mean = scale * s1[0] / double(k);
        result[0] = mean - 1.0;
        result[1] = mean;
        result[2] = scale * scale * s2[0] / double(k);
    }
}

cudaError_t launch_gather_xeb(const double2* acc, const int32_t* key_root, int64_t k, const RootMap& rm,
                              double2* amps, double* partials, int n_blocks, double* result, int n_qubits,
                              cudaStream_t st) {
    k_gather_xeb<<<n_blocks, 256, 0, st>>>(acc, key_root, k, rm, amps, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_xeb_final<<<1, 256, 0, st>>>(partials, n_blocks, k << rm.w, n_qubits, result);
    return cudaGetLastError();
}

cudaError_t prepare_tc_kernels();

cudaError_t prepare_kernels() {
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_trie_keys, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(size_t(kMaxTrieK) * 12));
    if (e != cudaSuccess) return e;
#define XEB_PREP_STREAM(T, P)                                                                            \
    e = cudaFuncSetAttribute(k_gemm_stream<T, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024); \
    if (e != cudaSuccess) return e;
    XEB_PREP_STREAM(float2, 1) XEB_PREP_STREAM(float2, 2) XEB_PREP_STREAM(float2, 4)
    XEB_PREP_STREAM(float2, 8) XEB_PREP_STREAM(float2, 16)
    XEB_PREP_STREAM(double2, 1) XEB_PREP_STREAM(double2, 2) XEB_PREP_STREAM(double2, 4)
    XEB_PREP_STREAM(double2, 8) XEB_PREP_STREAM(double2, 16)
#undef XEB_PREP_STREAM
    e = cudaFuncSetAttribute(k_gemm_kdeep<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(kdeep_smem_bytes<double2>()));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_gemm_memo<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_gemm_memo<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024);
    if (e != cudaSuccess) return e;
    e = prepare_tc_kernels();
    if (e != cudaSuccess) return e;
    done = true;
    return cudaSuccess;
}

// ---- instantiations ------------------------------------------------------------------
template cudaError_t launch_leaves<float2>(const LeafDesc*, int, const float2*, float2*, const char*, int64_t, cudaStream_t);
template cudaError_t launch_leaves<double2>(const LeafDesc*, int, const double2*, double2*, const char*, int64_t, cudaStream_t);
template cudaError_t launch_permute<float2>(const PermDesc&, const float2*, float2*, cudaStream_t);
template cudaError_t launch_permute<double2>(const PermDesc&, const double2*, double2*, cudaStream_t);
template cudaError_t launch_gemm<float2>(int, const GemmDesc&, float2*, cudaStream_t);
template cudaError_t launch_gemm<double2>(int, const GemmDesc&, double2*, cudaStream_t);
template cudaError_t launch_gemm_stream<float2>(const GemmDesc&, const StreamDesc&, float2*, cudaStream_t);
template cudaError_t launch_gemm_stream<double2>(const GemmDesc&, const StreamDesc&, double2*, cudaStream_t);
template cudaError_t launch_gemm_memo<float2>(const GemmDesc&, const StreamDesc&, float2*, char*, cudaStream_t);
template cudaError_t launch_gemm_memo<double2>(const GemmDesc&, const StreamDesc&, double2*, char*, cudaStream_t);
template cudaError_t launch_root_accum<float2>(const float2*, double2*, int64_t, cudaStream_t);
template cudaError_t launch_root_accum<double2>(const double2*, double2*, int64_t, cudaStream_t);

}  // namespace xebk
