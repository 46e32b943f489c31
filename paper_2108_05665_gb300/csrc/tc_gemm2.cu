// Split-precision complex contraction on tcgen05 with the small operand in
// tensor memory.
//
// The complex product C = A B is computed as the real product C' = A' W with
// W = [[Re B, Im B], [-Im B, Re B]] interleaved, in the operand roles
//
//     D (2N x rows) = W^T (2N x 2K) * A'^T (2K x rows)
//
// Split precision: every FP32 operand value x is split into x = big + small
// with small = RN_tf32(x - big), and D = big*big + big*small + small*big (+
// small*small with split_terms = 4).  big*big goes into its own FP32
// accumulator, the cross terms into another; the two are added with
// round-to-nearest in the epilogue.  The tensor cores truncate when they
// accumulate, which biases a long sum of products toward zero; over a chain of
// contractions that bias would shift every probability, and with it F, by
// many times the amplitude error.  So the big parts are not rounded per value:
// the bigs of one group -- one state row of one 32-float K-chunk, one row of
// W^T over all of K -- are the group's values rounded to the nearest multiple
// of the unit u = 2^(e - split_bits + 1), 2^e <= (largest |x| of the group) <
// 2^(e+1).  Each big is then an integer of at most split_bits bits times u
// (an exact TF32 value), every big*big product of one output element is an
// integer multiple of u_row * u_col, and their sum is exact in FP32 as long as
// it stays below 2^24 such units: no truncation happens.  The small parts
// carry the rest of each value to 11 more bits.
//
// W^T (big and small, <= 128 x 128 floats each) is written once per CTA into
// tensor memory and serves as the MMA's A operand; the state rows are the
// shared-memory B operand (K-major, 128-byte swizzle).  Gather mode: eight
// producer warps gather state elements (the k legs of a contraction sit at
// arbitrary address bits) with the loads of four chunks in flight per thread
// in registers, and write each chunk split into big/small into a ring stage.
// TMA mode (A row-major): one thread loads whole tiles with TMA boxes and four
// warps split them in place.  One thread issues the MMAs; the epilogue warps
// read D^T from tensor memory (lane = output column), release it to the next
// tile's MMAs, transpose the tile through an XOR-swizzled shared buffer and
// write C.
//
// Tensor memory: columns [0, 128) W^T big, [128, 256) W^T small, [256, 384)
// big*big accumulator, [384, 512) cross-term accumulator (128-row tiles: one
// MMA instruction covers 128 state rows).  Every wait is
// bounded (2 s, error word); the CTA always drains its MMAs and frees tensor
// memory before returning.
#include "kernels.cuh"
#include "tc_common.cuh"

namespace xebk {

namespace {

constexpr int kRows = 128;           // state rows per tile (UMMA N)
static_assert(kRows == 1 << kTc2RowBits, "tile rows must match the host tiling");
constexpr int kM = 128;              // W^T rows (UMMA M), N2 padded to 128
constexpr int kChunk = 32;           // floats of K' per chunk (one swizzle atom)
// Warp roles (14 warps).  Gather mode: warps 0-7 gather A, 8-11 epilogue.
// TMA mode: warps 0-3 split landed chunks, 4-11 epilogue (two warps per
// tensor-memory lane quarter, each with half the tile rows), 13 issues the
// TMA loads.  Warp 12 issues the MMAs in both modes.
constexpr int kMmaWarp = 12;
constexpr int kTmaWarp = 13;
constexpr int kThreads = 32 * 14;                 // 448
template <bool kTma>
__host__ __device__ constexpr int prod_warps() { return kTma ? 4 : 8; }
template <bool kTma>
__host__ __device__ constexpr int epi_warps() { return kTma ? 8 : 4; }
constexpr int kProd = 32 * 8;                     // gather mode: 256 producer threads
constexpr int kPerThread = kRows * 16 / kProd;    // gather mode: 8 complex elements per producer per chunk
constexpr int kLook = 4;                          // gather mode: chunks of loads in flight per producer (registers)
constexpr int kStageBytes = 2 * kRows * 128;      // operand stage: big + small, 16 KB each
constexpr int kSmallBytes = kRows * 128;          // TMA mode: stage of one chunk's small parts, 16 KB
constexpr int kRingGather = 4;                    // operand stages, gather mode
constexpr int kRingTma = 2;                       // small-part stages, TMA mode
constexpr int kRaw = 2;                           // whole-tile buffers, TMA mode
constexpr int kTileBytes = kRows * 128 * 4;       // TMA mode: one tile, 128 rows x up to 128 floats (64 KB)
constexpr int kCStride = 128;                     // floats per staged output row (XOR-swizzled columns)
constexpr uint32_t kTmemCols = 512;
template <bool kTma>
__host__ __device__ constexpr int op_stages() { return kTma ? kRingTma : kRingGather; }
template <bool kTma>
__host__ __device__ constexpr size_t ring_bytes() {
    return kTma ? size_t(kRaw) * kTileBytes + size_t(kRingTma) * kSmallBytes : size_t(kRingGather) * kStageBytes;
}

struct Sm2 {
    // rawb: gather mode, all producers have stored their raw values of a stage
    uint64_t full[kRingGather], empty[kRingGather], rawb[kRingGather], rfull[kRaw], rempty[kRaw], tfull[2], tempty[2],
        wready, drain, epi, never, pad_never;
    uint32_t tmem, pad;
    // staging offset (floats) of tile row r = rlo[r % 32] ^ rhi[r / 32]: the
    // row's base r * kCStride with its column swizzle folded in (linear in r)
    int32_t rlo[32], rhi[kRows / 32];
    // per result-tile bit i (ascending C order): C increment and staging-slot
    // XOR; per tile index bit outside the tile: C increment
    int64_t cinc[16];
    int32_t sinc[16];
    int64_t extinc[32];
};

}  // namespace

template <bool kTma, bool kGrp>
__global__ void __launch_bounds__(kThreads, 1)
    k_tc_gemm2(const __grid_constant__ TcDesc t, const __grid_constant__ CUtensorMap tmap, float2* __restrict__ arena) {
    constexpr int kRing = op_stages<kTma>();
    constexpr int kProdWarps = prod_warps<kTma>();
    constexpr int kProdT = 32 * kProdWarps;        // threads that fill the operand ring
    constexpr int kEpiWarps = epi_warps<kTma>();
    constexpr int kEpiWarp0 = kProdWarps;
    constexpr int kEpiT = 32 * kEpiWarps;
    extern __shared__ __align__(1024) unsigned char raw2[];
    // 1024-byte aligned base, derived from the shared array by pointer
    // arithmetic so every pointer below stays a shared-memory pointer
    unsigned char* sm = raw2 + ((1024u - (smem_u32(raw2) & 1023u)) & 1023u);
    // TMA mode: kRaw whole-tile buffers (raw values, split in place into the
    // bigs), then kRingTma stages of one chunk's smalls.  Gather mode: kRing
    // stages of (big 16 KB | small 16 KB).
    unsigned char* tbuf = sm;
    unsigned char* ring = sm + (kTma ? kRaw * kTileBytes : 0);
    float* cst = reinterpret_cast<float*>(sm + ring_bytes<kTma>());  // kRows x kCStride
    Sm2* S = reinterpret_cast<Sm2*>(cst + kRows * kCStride);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t n_tiles = kGrp ? t.n_groups * t.tpg : t.M / kRows;
    // tiles of this CTA: t_first, t_first + t_step, ... below t_end.  Keyed
    // mode takes one contiguous block, so consecutive tiles mostly share their
    // key and W^T is rewritten about once per key; the other modes take every
    // gridDim.x-th tile.
    const bool blocked = kGrp && t.keyed;
    const int64_t per_cta = (n_tiles + gridDim.x - 1) / gridDim.x;
    const int64_t t_first = blocked ? int64_t(blockIdx.x) * per_cta : int64_t(blockIdx.x);
    const int64_t t_end = blocked ? (t_first + per_cta < n_tiles ? t_first + per_cta : n_tiles) : n_tiles;
    const int64_t t_step = blocked ? 1 : int64_t(gridDim.x);
    const int64_t my_tiles = t_end > t_first ? (t_end - 1 - t_first) / t_step + 1 : 0;
    const int nch = t.n_chunks;
    if (tid == 0) {
        for (int s = 0; s < kRing; ++s) {
            bar_init(&S->full[s], kProdT);
            bar_init(&S->empty[s], 1);
            bar_init(&S->rawb[s], kProdT);
        }
        for (int s = 0; s < kRaw; ++s) {
            bar_init(&S->rfull[s], 1);
            bar_init(&S->rempty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            bar_init(&S->tfull[b], 1);
            bar_init(&S->tempty[b], kEpiT);
        }
        bar_init(&S->wready, kEpiT);
        bar_init(&S->drain, 1);
        bar_init(&S->never, 1);
        bar_init(&S->epi, kEpiT);
    }
    if (tid < 32 + kRows / 32) {
        // x(r): XOR of the swizzle vectors of r's bits (tile row bit b is
        // tile bit i with st_is_n clear and st_idx = b)
        const int r = tid < 32 ? tid : (tid - 32) * 32;
        int x = 0;
        for (int i = 0; i < t.Tst; ++i)
            if (!((t.st_is_n >> i) & 1) && ((r >> t.st_idx[i]) & 1)) x ^= int(t.st_swz[i]);
        (tid < 32 ? S->rlo[tid] : S->rhi[tid - 32]) = (r * kCStride) ^ (2 * x);
    }
    if (tid < 16) {
        const int i = tid;
        S->cinc[i] = i < t.Tst ? int64_t(1) << t.st_pos[i] : 0;
        S->sinc[i] = i < t.Tst ? ((((t.st_is_n >> i) & 1) ? (1 << t.st_idx[i]) : (1 << t.st_idx[i]) * (kCStride / 2)) ^
                                  int(t.st_swz[i]))
                               : 0;
    }
    if (tid >= 32 && tid < 64) {
        const int i = tid - 32;
        S->extinc[i] = i < t.n_ext ? int64_t(1) << t.ext_cpos[i] : 0;
    }
    if (tid == 0) {
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S->tmem)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = S->tmem;
    const uint32_t w_big = tmem, w_small = tmem + 128;

    if (kTma && warp < kProdWarps) {
        // ---------------- TMA mode: split each landed tile, chunk by chunk ----------------
        // A tile lands as 16 groups of 8 consecutive A rows, each group holding
        // all of its rows' chunks: group j, chunk c is the 1024-byte swizzle
        // atom at j * (n_chunks KB) + c KB, 128-byte line per row -- the
        // layout the MMA reads with an 8-row-group stride of n_chunks KB.
        // Thread tid splits tile row tid: its line of chunk c gives the row's
        // grid; the bigs overwrite the raw values in place, the smalls go to a
        // small-part stage at the same position inside a contiguous tile
        // (group stride 1 KB).  16-byte units are visited from (tid & 7) on,
        // so the 8 lanes of each shared-memory phase touch 8 bank groups.
        static_assert(!kTma || kProdT == kRows, "one split thread per tile row");
        const int gsz = nch * 1024;
        int64_t g = 0;
        bool ok = true;
        for (int64_t i = 0; i < my_tiles && ok; ++i) {
            const int b = int(i & 1);
            if (!bar_wait(&S->rfull[b], uint32_t(i >> 1) & 1, t.err, 20, t.wait_ns)) break;
            unsigned char* rowp = tbuf + b * kTileBytes + (tid >> 3) * gsz + (tid & 7) * 128;
            for (int c = 0; c < nch; ++c, ++g) {
                const int s2 = int(g & 1);
                unsigned char* src = rowp + c * 1024;
                float4 v[8];
                float m = 0.f;
#pragma unroll
                for (int i2 = 0; i2 < 8; ++i2) {
                    v[i2] = *reinterpret_cast<const float4*>(src + 16 * ((i2 + tid) & 7));
                    m = fmaxf(m, absmax4(v[i2]));
                }
                const float cg = grid_c(m, t.split_bits);
                if (!bar_wait(&S->empty[s2], (uint32_t(g >> 1) & 1) ^ 1, t.err, 11, t.wait_ns)) {
                    ok = false;
                    break;
                }
                unsigned char* ds = ring + s2 * kSmallBytes + (tid >> 3) * 1024 + (tid & 7) * 128;
#pragma unroll
                for (int i2 = 0; i2 < 8; ++i2) {
                    float4 bg, sm4;
                    split4(v[i2], cg, bg, sm4);
                    *reinterpret_cast<float4*>(src + 16 * ((i2 + tid) & 7)) = bg;
                    *reinterpret_cast<float4*>(ds + 16 * ((i2 + tid) & 7)) = sm4;
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                bar_arrive(&S->full[s2]);
            }
        }
    } else if (kTma && warp == kTmaWarp) {
        // ---------------- TMA mode: one thread loads whole tiles ----------------
        // 16 boxes per tile, each 8 consecutive A rows x all chunks: every box
        // reads 8 whole rows (8 x n_chunks x 128 contiguous bytes)
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmap)) : "memory");
            const int nbox = kRows >> 3;
            const int gsz = nch * 1024;
            auto ybase = [&](int64_t tile) {
                int64_t y = 0;
                for (int i = 0; i < t.n_ext; ++i)
                    if ((tile >> i) & 1) y |= int64_t(1) << (t.ext_apos[i] - t.row_shift);
                return y;
            };
            int64_t i = 0;
            for (int64_t tile = t_first; tile < t_end; tile += t_step, ++i) {
                const int b = int(i & 1);
                if (!bar_wait(&S->rempty[b], (uint32_t(i >> 1) & 1) ^ 1, t.err, 18, t.wait_ns)) break;
                bar_expect_tx(&S->rfull[b], uint32_t(kRows * 128 * nch));
                const int64_t y0 = ybase(tile);
                unsigned char* dst = tbuf + b * kTileBytes;
                for (int j = 0; j < nbox; ++j)
                    tma_load_3d(dst + j * gsz, &tmap, 0, int(y0 + t.box_y[j]), 0, &S->rfull[b]);
            }
            // the CTA must not exit with copies in flight: wait (bounded) for the last ones
            for (int64_t d = i > kRaw ? i - kRaw : 0; d < i; ++d)
                bar_wait_drain(&S->rfull[d % kRaw], uint32_t(d / kRaw) & 1, t.wait_ns);
        }
        __syncwarp();
    } else if (!kTma && warp < kProdWarps) {
        // ---------------- producers: gather into registers, split into the ring ----------------
        // Each thread keeps the loads of kLook chunks in flight in registers.
        // Chunk c is stored raw into the big half of its ring stage once the
        // stage is free, then the loads of chunk c + kLook are issued.  When
        // all producers have stored theirs (rawb), thread tid splits half
        // (tid & 1) of tile row tid >> 1 in place: the row's grid needs all of
        // its 32 values, which other threads loaded.
        int32_t off[kPerThread];
        uint32_t pos[kPerThread];
#pragma unroll
        for (int j = 0; j < kPerThread; ++j) {
            const int e = tid + kProd * j;
            int r = 0, k = 0, ri = 0, ki = 0;
            int32_t o = 0;
            for (int i = 0; i < t.T; ++i) {
                const int bit = (e >> i) & 1;
                if ((t.is_k >> i) & 1) k |= bit << ki++;
                else r |= bit << ri++;
                if (bit) o |= int32_t(1) << t.pos[i];
            }
            off[j] = o;
            pos[j] = swz(uint32_t(r) * 128u + uint32_t(k) * 8u);
        }
        const int64_t total = my_tiles * nch;
        // issue-side cursor (chunks are issued in order)
        int64_t ld_tile = t_first;
        int ld_c = 0;
        int64_t cg = -1, cga = 0;   // grouped mode: last group seen and its A offset
        auto tile_base = [&](int64_t tile) {
            int64_t b = 0;
            if constexpr (kGrp) {
                const int64_t g = tile / t.tpg;
                tile -= g * t.tpg;
                if (g != cg) {
                    cg = g;
                    cga = t.keyed ? (t.uL ? int64_t(t.uL[g]) * t.a_key : 0) : t.grp_a[g];
                }
                b = cga;
            }
            for (int i = 0; i < t.n_ext; ++i)
                if ((tile >> i) & 1) b += int64_t(1) << t.ext_apos[i];
            return b;
        };
        const float2* Arow = arena + t.a_off + tile_base(ld_tile) + t.chunk_off[0];
        float2 buf[kLook][kPerThread];
#define XEB_TC2_ISSUE(U)                                                                   \
    do {                                                                                   \
        _Pragma("unroll") for (int j = 0; j < kPerThread; ++j) buf[U][j] = __ldg(Arow + off[j]); \
        if (++ld_c == nch) {                                                               \
            ld_c = 0;                                                                      \
            ld_tile += t_step;                                                             \
            Arow = arena + t.a_off + (ld_tile < t_end ? tile_base(ld_tile) : 0) + t.chunk_off[0]; \
        } else {                                                                           \
            Arow += t.chunk_off[ld_c] - t.chunk_off[ld_c - 1];                             \
        }                                                                                  \
    } while (0)
#pragma unroll
        for (int u = 0; u < kLook; ++u)
            if (u < total) XEB_TC2_ISSUE(u);
        static_assert(kTma || kProdT == 2 * kRows, "two producer threads per tile row in the split phase");
        const int prow = tid >> 1, phalf = tid & 1;
        bool ok = true;
        for (int64_t c0 = 0; c0 < total && ok; c0 += kLook) {
#pragma unroll
            for (int u = 0; u < kLook; ++u) {
                const int64_t c = c0 + u;
                if (c < total && ok) {
                    const int s = int(c % kRing);
                    const uint32_t use = uint32_t(c / kRing);
                    ok = __all_sync(0xffffffffu, bar_wait(&S->empty[s], (use & 1) ^ 1, t.err, 11, t.wait_ns));
                    if (ok) {
                        unsigned char* sb = ring + s * kStageBytes;
#pragma unroll
                        for (int j = 0; j < kPerThread; ++j) *reinterpret_cast<float2*>(sb + pos[j]) = buf[u][j];
                        bar_arrive(&S->rawb[s]);
                        ok = __all_sync(0xffffffffu, bar_wait(&S->rawb[s], use & 1, t.err, 19, t.wait_ns));
                    }
                    if (ok) {
                        unsigned char* sb = ring + s * kStageBytes;
                        // (values are read twice rather than held: the
                        // registers hold the loads in flight)
                        float m = 0.f;
#pragma unroll 1
                        for (int i = 0; i < 4; ++i)
                            m = fmaxf(m, absmax4(*reinterpret_cast<const float4*>(
                                             sb + swz(uint32_t(prow * 128 + phalf * 64 + 16 * i)))));
                        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 1));
                        const float cg = grid_c(m, t.split_bits);
#pragma unroll 1
                        for (int i = 0; i < 4; ++i) {
                            const uint32_t o = swz(uint32_t(prow * 128 + phalf * 64 + 16 * i));
                            float4 b, sm4;
                            split4(*reinterpret_cast<const float4*>(sb + o), cg, b, sm4);
                            *reinterpret_cast<float4*>(sb + o) = b;
                            *reinterpret_cast<float4*>(sb + kRows * 128 + o) = sm4;
                        }
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        bar_arrive(&S->full[s]);
                        if (c + kLook < total) XEB_TC2_ISSUE(u);
                    }
                }
            }
        }
#undef XEB_TC2_ISSUE
    } else if (warp == kMmaWarp) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(kRows >> 3) << 17) |
                                   (uint32_t(kM >> 4) << 24);
            bool ok = bar_wait(&S->wready, 0, t.err, 12, t.wait_ns);
            // testing aid (xeb_plan_test_wait): a wait that runs out -- nothing
            // arrives on `never` -- records a timeout, and every role then
            // leaves its loop as after any failed wait
            if (t.test_wait) ok = bar_wait(&S->never, 0, t.err, 30, t.wait_ns) && false;
            const bool four = t.split_terms == 4;
            fence_after();
            uint32_t it = 0, tc = 0;
            for (int64_t tile = t_first; tile < t_end && ok; tile += t_step, ++tc) {
                const uint32_t b = 0, ub = tc;  // one accumulator pair (TMEM is full)
                if (!bar_wait(&S->tempty[b], (ub & 1) ^ 1, t.err, 13, t.wait_ns)) break;
                fence_after();
                const uint32_t d_big = tmem + 256, d_small = d_big + kRows;
                for (int ch = 0; ch < nch; ++ch, ++it) {
                    const int s = int(it % kRing);
                    const uint32_t use = it / kRing;
                    if (!bar_wait(&S->full[s], use & 1, t.err, 14, t.wait_ns)) { ok = false; break; }
                    fence_after();
                    // big and small operands of this chunk (TMA mode: bigs in the
                    // tile buffer, 8-row groups n_chunks KB apart)
                    uint32_t sb, ss, sbo_b;
                    if constexpr (kTma) {
                        sb = smem_u32(tbuf + (tc & 1) * kTileBytes + ch * 1024);
                        ss = smem_u32(ring + s * kSmallBytes);
                        sbo_b = uint32_t(nch * 1024);
                    } else {
                        sb = smem_u32(ring + s * kStageBytes);
                        ss = sb + kRows * 128;
                        sbo_b = 1024;
                    }
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks) {
                        const uint32_t kc = uint32_t(ch * kChunk + ks * 8);  // TMEM column of this K step
                        const uint32_t kb = ks * 32;                          // byte offset in the swizzle atom
                        mma_ts(d_big, w_big + kc, sdesc(sb + kb, sbo_b), idesc, (ch | ks) != 0);
                        mma_ts(d_small, w_small + kc, sdesc(sb + kb, sbo_b), idesc, (ch | ks) != 0);
                        mma_ts(d_small, w_big + kc, sdesc(ss + kb), idesc, 1);
                        if (four) mma_ts(d_small, w_small + kc, sdesc(ss + kb), idesc, 1);
                    }
                    mma_commit(&S->empty[s]);
                }
                if (kTma && ok) mma_commit(&S->rempty[tc & 1]);   // the tile buffer is read
                if (!ok) break;
                mma_commit(&S->tfull[b]);
            }
            mma_commit(&S->drain);
            bar_wait(&S->drain, 0, t.err, 15, t.wait_ns);
        }
        __syncwarp();
    } else if (warp >= kEpiWarp0 && warp < kEpiWarp0 + kEpiWarps) {
        // ---------------- W^T into tensor memory, then the epilogue ----------------
        const int widx = warp - kEpiWarp0;       // 0 .. kEpiWarps - 1
        const int q = warp & 3;                  // tensor-memory lane quarter of this warp
        const int half = widx >> 2;              // which share of columns / rows
        constexpr int kShares = kEpiWarps / 4;
        const int np = q * 32 + lane;            // W^T row = output column n' (0..127)
        // W^T (big, small) of the columns of `tile` into tensor memory; in
        // grouped mode the columns are the keys of the tile's group
        auto write_wt = [&](int64_t tile) {
            const int n = np >> 1, cpart = np & 1;
            bool live = np < t.N2;
            const float2* B = arena + t.b_off;
            if constexpr (kGrp) {
                const int64_t g = tile / t.tpg;
                if (t.keyed) {   // key g's own B operand, all N columns
                    B = arena + t.b_off + (t.uR ? int64_t(t.uR[g]) * t.b_key : 0);
                } else {
                    const int64_t u0 = t.gstart[g];
                    live = np < 2 * (t.gstart[g + 1] - u0);
                    B = arena + t.bpack_off + u0 * (t.K2 / 2);
                }
            }
            int64_t noff = 0;
            if (live)
                for (int i = 0; i < t.nbn; ++i)
                    if ((n >> i) & 1) noff |= int64_t(1) << t.bpn[i];
            // value kp of this W^T row: Re / Im of B[k][n] with the sign of
            // the real expansion (0 for padding rows)
            auto wval = [&](int kp) {
                const int k = kp >> 1, apart = kp & 1;
                if (!live) return 0.f;
                int64_t off = noff;
                for (int b = 0; b < t.nbk; ++b)
                    if ((k >> b) & 1) off |= int64_t(1) << t.bpk[b];
                const float2 bv = B[off];
                return cpart == 0 ? (apart == 0 ? bv.x : -bv.y) : (apart == 0 ? bv.y : bv.x);
            };
            // the row's grid: its largest magnitude over all of K (32 loads in
            // flight per step)
            float wm = 0.f;
            for (int c0 = 0; c0 < t.K2; c0 += 32) {
#pragma unroll
                for (int i = 0; i < 32; ++i) wm = fmaxf(wm, fabsf(wval(c0 + i)));
            }
            const float cw = grid_c(wm, t.split_bits);
            for (int c0 = 32 * half; c0 < t.K2; c0 += 32 * kShares) {
                float vb[32], vs[32];
#pragma unroll
                for (int i = 0; i < 32; ++i) split_on(wval(c0 + i), cw, vb[i], vs[i]);
                const uint32_t lanes = uint32_t(q * 32) << 16;
                tm_st32(w_big + lanes + uint32_t(c0), vb);
                tm_st32(w_small + lanes + uint32_t(c0), vs);
            }
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        };
        if (t_first < t_end) write_wt(t_first);
        fence_before();
        bar_arrive(&S->wready);
        uint32_t tc = 0, ep = 0;
        const uint32_t lanes = uint32_t(q * 32) << 16;
        // Result tile element e (its bits in ascending C address order) =
        // h * 32 + lane.  Its C offset and staging slot are sums of one
        // increment per set bit, so each warp owns a contiguous block of h and
        // keeps the increments of the block's low 3 bits in registers: eight
        // independent staging loads and stores per group, no table lookups.
        auto ginc = [&](int i) { return int64_t(1) << t.st_pos[i]; };
        // staging slot (float2 units) of tile bit i: row r -> r * 64, column
        // n -> n, each XOR its swizzle vector; slots combine by XOR
        auto sinc = [&](int i) {
            return (((t.st_is_n >> i) & 1) ? (1 << t.st_idx[i]) : (1 << t.st_idx[i]) * (kCStride / 2)) ^
                   int(t.st_swz[i]);
        };
        // staging writes: the swizzle of each tile row bit, and the XOR of
        // the swizzles of this thread's column bits (>= 4: one per warp)
        int xn = 0;
        for (int i = 0; i < t.Tst; ++i)
            if (((t.st_is_n >> i) & 1) && (((np >> 1) >> t.st_idx[i]) & 1)) xn ^= int(t.st_swz[i]);
        const int npx = np ^ (2 * xn);   // this thread's swizzled staging column
        int lo_slot = 0;
        int64_t lo_glob = 0;
        for (int i = 0; i < 5; ++i)  // Tst >= 11 (7 row bits + >= 4 column bits)
            if ((lane >> i) & 1) {
                lo_glob += ginc(i);
                lo_slot ^= sinc(i);
            }
        constexpr int kWB = kEpiWarps == 8 ? 3 : 2;  // log2(epilogue warps)
        const int hb = t.Tst - 5;                    // bits of h
        const int qb = hb < kWB ? hb : kWB;          // bits selecting the warp's block
        const int wb = hb - qb;                      // bits inside the block
        const int lb = wb < 3 ? wb : 3;              // of which held in registers
        const bool e_active = widx < (1 << qb);
        int64_t gq = lo_glob;
        int sq = lo_slot;
        for (int i = 0; i < qb; ++i)
            if ((widx >> i) & 1) {
                gq += ginc(5 + wb + i);
                sq ^= sinc(5 + wb + i);
            }
        int64_t g8[8];
        int s8[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            g8[j] = 0;
            s8[j] = 0;
            for (int b = 0; b < lb; ++b)
                if ((j >> b) & 1) {
                    g8[j] += ginc(5 + b);
                    s8[j] ^= sinc(5 + b);
                }
        }
        const int nlo = 1 << lb, nmid = 1 << (wb - lb);
        // the middle loop's bits are tile bits 5 + lb .. 4 + wb (at most 6:
        // Tst <= 16); their increments and those of the tile index bits
        // outside the tile come from the shared tables (no parameter array
        // is indexed inside the tile loop)
        const int jb0 = 5 + lb;
        // bounded sync of the four epilogue warps (an aborting warp cannot
        // leave the others blocked)
        auto epi_sync = [&]() {
            bar_arrive(&S->epi);
            const bool ok = bar_wait(&S->epi, ep & 1, t.err, 17, t.wait_ns);
            ++ep;
            return ok;
        };
        for (int64_t tile = t_first; tile < t_end; tile += t_step, ++tc) {
            const uint32_t b = 0, ub = tc;
            const bool got = bar_wait(&S->tfull[b], ub & 1, t.err, 16, t.wait_ns);
            if (!__all_sync(0xffffffffu, got)) break;
            fence_after();
            // grouped mode: the next tile of this CTA needs its group's W^T,
            // written after this tile's accumulators are read and before they
            // are released (the MMAs of this tile are complete by then)
            const int64_t nxt = tile + t_step;
            const bool switch_w = kGrp && nxt < t_end && nxt / t.tpg != tile / t.tpg;
            // D^T: lane = output column np, column = tile row; tensor memory is
            // released for the next tile's MMAs once the last load has landed
            const uint32_t db = tmem + 256;
            constexpr int kMyRows = kRows / kShares;
            // staging slots of a 32-row chunk of this thread's column
            auto stage = [&](int r0, const float* x) {
                const int cb = S->rhi[r0 >> 5] ^ npx;
#pragma unroll
                for (int i = 0; i < 32; i += 4) {
                    const int4 ro = *reinterpret_cast<const int4*>(&S->rlo[i]);
                    cst[ro.x ^ cb] = x[i];
                    cst[ro.y ^ cb] = x[i + 1];
                    cst[ro.z ^ cb] = x[i + 2];
                    cst[ro.w ^ cb] = x[i + 3];
                }
            };
            if constexpr (kMyRows == 64) {
                // both 32-row chunks of this warp are read and summed first, so
                // the accumulators go back to the MMAs before any staging write
                const int r0 = half * kMyRows;
                float v0[32], v1[32], w[16];
                tm_ld32(db + lanes + uint32_t(r0), v0);
                tm_ld32(db + lanes + uint32_t(r0 + 32), v1);
#pragma unroll
                for (int h = 0; h < 64; h += 16) {   // the cross-term accumulator, 16 columns at a time
                    tm_ld16(db + lanes + kRows + uint32_t(r0 + h), w);
                    tm_wait_ld();
                    if (h == 48 && !switch_w) {
                        fence_before();
                        bar_arrive(&S->tempty[b]);
                    }
                    float* x = h < 32 ? v0 + h : v1 + (h - 32);
#pragma unroll
                    for (int i = 0; i < 16; ++i) x[i] += w[i];
                }
                stage(r0, v0);
                stage(r0 + 32, v1);
            } else {
                for (int r0 = half * kMyRows; r0 < (half + 1) * kMyRows; r0 += 32) {
                    float v[32], w[32];
                    tm_ld32(db + lanes + uint32_t(r0), v);
                    tm_ld32(db + lanes + kRows + uint32_t(r0), w);
                    tm_wait_ld();
                    if (r0 == (half + 1) * kMyRows - 32 && !switch_w) {
                        fence_before();
                        bar_arrive(&S->tempty[b]);
                    }
                    const int cb = S->rhi[r0 >> 5] ^ npx;
#pragma unroll
                    for (int i = 0; i < 32; i += 4) {
                        const int4 ro = *reinterpret_cast<const int4*>(&S->rlo[i]);
                        cst[ro.x ^ cb] = v[i] + w[i];
                        cst[ro.y ^ cb] = v[i + 1] + w[i + 1];
                        cst[ro.z ^ cb] = v[i + 2] + w[i + 2];
                        cst[ro.w ^ cb] = v[i + 3] + w[i + 3];
                    }
                }
            }
            if (switch_w) {
                write_wt(nxt);
                fence_before();
                bar_arrive(&S->tempty[b]);
            }
            if (!__all_sync(0xffffffffu, epi_sync())) break;
            int64_t cbase = 0, mt = tile;
            int nk = 1 << 30;   // grouped mode: keys (columns) of this tile's group
            if constexpr (kGrp) {
                const int64_t g = tile / t.tpg;
                mt = tile - g * t.tpg;
                if (t.keyed) {   // key g's result block
                    cbase = g * t.c_key;
                } else {
                    const int64_t u0 = t.gstart[g];
                    nk = int(t.gstart[g + 1] - u0);
                    cbase = u0 * t.c_key;
                }
            }
            {   // C offset of the tile index bits outside the tile: one bit per lane, summed
                int64_t xb = ((mt >> lane) & 1) ? S->extinc[lane] : 0;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) xb += __shfl_xor_sync(0xffffffffu, xb, o);
                cbase += xb;
            }
            float2* C = arena + t.c_off + cbase;
            const float2* st2 = reinterpret_cast<const float2*>(cst);
            if (e_active && (!kGrp || t.keyed)) {
                for (int jm = 0; jm < nmid; ++jm) {
                    int64_t gm = gq;
                    int sm2 = sq;
                    for (int bb = 0; (jm >> bb) != 0; ++bb)
                        if ((jm >> bb) & 1) {
                            gm += S->cinc[jb0 + bb];
                            sm2 ^= S->sinc[jb0 + bb];
                        }
                    float2 v[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        if (j < nlo) v[j] = st2[sm2 ^ s8[j]];
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        if (j < nlo) C[gm + g8[j]] = v[j];
                }
            } else if (e_active) {   // grouped mode: only the group's nk key columns exist
                for (int jm = 0; jm < nmid; ++jm) {
                    int64_t gm = gq;
                    int sm2 = sq;
                    for (int bb = 0; (jm >> bb) != 0; ++bb)
                        if ((jm >> bb) & 1) {
                            gm += S->cinc[jb0 + bb];
                            sm2 ^= S->sinc[jb0 + bb];
                        }
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        if (j < nlo && ((sm2 ^ s8[j]) & (kCStride / 2 - 1)) < nk) C[gm + g8[j]] = st2[sm2 ^ s8[j]];
                }
            }
            if (!__all_sync(0xffffffffu, epi_sync())) break;
        }
    }
    fence_before();
    __syncthreads();
    if (warp == kMmaWarp) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

// 1024 bytes of alignment slack + rings + output staging + barriers/tables
template <bool kTma>
constexpr size_t tc2_smem() {
    return 1024 + ring_bytes<kTma>() + size_t(kRows) * kCStride * 4 + sizeof(Sm2);
}
static_assert(offsetof(Sm2, rlo) % 16 == 0, "row table read as int4");
static_assert(sizeof(Sm2) % 8 == 0 && tc2_smem<true>() <= 232448 && tc2_smem<false>() <= 232448,
              "tensor-memory contraction exceeds the shared memory of one CTA");

cudaError_t prepare_tc_kdeep();

cudaError_t prepare_tc_kernels() {
    cudaError_t e = prepare_tc_kdeep();
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_tc_gemm2<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(tc2_smem<true>()));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_tc_gemm2<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(tc2_smem<false>()));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_tc_gemm2<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(tc2_smem<false>()));
}

cudaError_t launch_tc_gemm2(const TcDesc& t, const CUtensorMap& tmap, float2* arena, int n_sms, cudaStream_t st) {
    const int64_t tiles = t.grp ? t.n_groups * t.tpg : t.M / kRows;
    const int grid = int(tiles < n_sms ? tiles : n_sms);
    if (t.tma)
        k_tc_gemm2<true, false><<<grid, kThreads, tc2_smem<true>(), st>>>(t, tmap, arena);
    else if (t.grp)
        k_tc_gemm2<false, true><<<grid, kThreads, tc2_smem<false>(), st>>>(t, tmap, arena);
    else
        k_tc_gemm2<false, false><<<grid, kThreads, tc2_smem<false>(), st>>>(t, tmap, arena);
    return cudaGetLastError();
}

}  // namespace xebk
