// Keyed contractions with a deep summed index on tcgen05 (split precision).
//
// C_u = A_uL(u) (M x K) * B_uR(u) (K x N) for every key u of a keyed
// contraction (App. A: 2^(q+r) multiply-adds per key), M, N in {16, 32}
// complex, K a multiple of 64 complex.  These are the contractions near the
// root of sliced plans: each key owns a small result and sums thousands of
// terms.
//
// Real expansion and split as in tc_gemm2.cu: per key D (2N x M) = W^T (2N x
// 2K) * A'^T (2K x M), W = [[Re B, Im B], [-Im B, Re B]] interleaved; every
// value is split into a TF32 big part on a common grid (one grid per row of a
// 32-float K-chunk: a row of A', a row of W^T) and a TF32 small part; big*big
// and big*small + small*big + small*small go to separate FP32 accumulators.
//
// Keys are stacked block-diagonally: KPM = 128 / (2N) keys per MMA, W^T of key
// j in rows 2N j .. 2N (j+1) - 1 of a 128-row operand, A'^T of key j in rows
// M j .. M (j+1) - 1 of an NM = KPM M row operand, so one MMA (M = 128, N =
// NM, K = 8) computes every key's product in the diagonal blocks of D (the
// rest of D is never read).  Any KPM consecutive keys share an MMA; keys that
// share a left key mostly sit next to each other (keys are ordered by left
// key), so their A rows come from L2.  Both operands are in shared memory,
// per K-chunk of 16 complex (32 floats = one 128-byte swizzle line per row):
//
//   W^T big | W^T small (128 rows each) | A'^T big | A'^T small (NM rows each)
//
// Exactness of the big*big sums needs them to stay below 2^24 grid units, so
// the big*big chain restarts every 4 chunks (K' = 128, as in tc_gemm2.cu) in
// one of two tensor-memory accumulators (ping-pong); the epilogue adds each
// finished segment to FP32 registers with round-to-nearest while the MMAs run
// on into the other one.  The cross terms use one accumulator per key block
// (two, ping-pong across blocks).
//
// Warps: 0-3 load the operands (plain loads: the legs sit at arbitrary
// address bits) and split them into the stage ring; 4-7 are the epilogue
// (warp 4 + q owns tensor-memory lanes 32q .. 32q + 31, i.e. rows of key
// 32q / 2N); warp 8 issues the MMAs.  Every wait is bounded (opts.timeout_ms,
// error word); the CTA drains its MMAs and frees tensor memory before it
// returns.
#include "kernels.cuh"
#include "tc_common.cuh"

namespace xebk {

namespace {

constexpr int kKdThreads = 32 * 9;
constexpr int kKdLoadT = 128;       // loader threads (warps 0-3)
constexpr int kKdEpiWarp0 = 4;
constexpr int kKdMmaWarp = 8;
constexpr int kWBytes = 128 * 128;  // 128 W^T rows x 32 floats
constexpr int kSeg = 4;             // chunks per big*big segment (K' = 128)

template <int M, int N>
struct KdShape {
    static constexpr int KPM = 128 / (2 * N);             // keys per MMA
    static constexpr int NM = KPM * M;                    // A'^T rows = MMA N
    static constexpr int ABytes = NM * 128;
    static constexpr int StageBytes = 2 * kWBytes + 2 * ABytes;
    // raw values each loader thread has in flight per chunk (cp.async, 8 bytes each)
    static constexpr int PerThread = (NM * 4 / 128 + KPM * N * 4 / 128) * 4;
    static constexpr int RawBytes = PerThread * 128 * 8;     // one chunk, all loader threads
    static constexpr int Stages = 2;
    static constexpr int RawDepth = (200 * 1024 - Stages * StageBytes) / RawBytes < 6
                                        ? (200 * 1024 - Stages * StageBytes) / RawBytes
                                        : 6;                  // chunks of raw loads in flight
    // bb ping-pong + cross ping-pong, NM columns each (a power of two >= 32)
    static constexpr uint32_t TmemCols = 4 * NM <= 128 ? 128 : 4 * NM <= 256 ? 256 : 512;
    static_assert(NM % 16 == 0 && NM <= 128, "MMA N of the stacked keys");
    static_assert(RawDepth >= 2, "raw ring");
};

constexpr int kMaxStages = 8;
constexpr int kMaxChunks = 512;     // K <= 8192 complex
struct SmKd {
    uint64_t full[kMaxStages], empty[kMaxStages], segfull[2], segempty[2], crfull[2], crempty[2], drain, never;
    uint32_t tmem, pad;
    int64_t cm[32];                 // C offset of result row m
    int64_t cka[kMaxChunks], ckb[kMaxChunks];   // A / B offset of K-chunk c (k bits >= 4)
};

__device__ __forceinline__ int64_t scat(int64_t x, const int8_t* pos, int n) {
    int64_t o = 0;
    for (int i = 0; i < n; ++i)
        if ((x >> i) & 1) o |= int64_t(1) << pos[i];
    return o;
}

// swizzled byte offset of 16-byte unit u of 128-byte row r (1024-byte atoms)
__device__ __forceinline__ uint32_t kd_unit(int r, int u) { return uint32_t(r * 128 + ((u ^ (r & 7)) << 4)); }

// 8-byte asynchronous global -> shared copy; n = 0 fills zeros (src unread)
__device__ __forceinline__ void cp_async8(void* dst, const void* src, bool n) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(n ? 8 : 0)
                 : "memory");
}

// 32 lanes x 16 columns of tensor memory into registers (no wait)
__device__ __forceinline__ void tm_ld16(uint32_t ta, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(ta));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

template <int M>
__device__ __forceinline__ void tm_ldM(uint32_t ta, float* v) {
    if constexpr (M == 16) tm_ld16(ta, v);
    else tm_ld32(ta, v);
}

}  // namespace

template <int M, int N>
__global__ void __launch_bounds__(kKdThreads, 1)
    k_tc_kdeep(const __grid_constant__ KdDesc t, float2* __restrict__ arena) {
    using Sh = KdShape<M, N>;
    constexpr int KPM = Sh::KPM, NM = Sh::NM, kStages = Sh::Stages;
    extern __shared__ __align__(1024) unsigned char kd_raw[];
    unsigned char* sm = kd_raw + ((1024u - (smem_u32(kd_raw) & 1023u)) & 1023u);
    SmKd* S = reinterpret_cast<SmKd*>(sm + kStages * Sh::StageBytes + Sh::RawDepth * Sh::RawBytes);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nch = t.K / 16;               // K-chunks per key
    const int nseg = nch / kSeg;
    // this CTA's key blocks (KPM consecutive keys each)
    const int64_t n_blocks = (t.kv + KPM - 1) / KPM;
    const int64_t per = (n_blocks + gridDim.x - 1) / gridDim.x;
    const int64_t b_first = int64_t(blockIdx.x) * per;
    const int64_t b_end = b_first + per < n_blocks ? b_first + per : n_blocks;
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            bar_init(&S->full[s], kKdLoadT);
            bar_init(&S->empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            bar_init(&S->segfull[b], 1);
            bar_init(&S->segempty[b], 128);
            bar_init(&S->crfull[b], 1);
            bar_init(&S->crempty[b], 128);
        }
        bar_init(&S->drain, 1);
        bar_init(&S->never, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (tid < 32) S->cm[tid] = tid < M ? scat(tid, t.cpm, M == 16 ? 4 : 5) : 0;
    for (int c = tid; c < nch; c += kKdThreads) {
        S->cka[c] = scat(int64_t(c) << 4, t.apk, t.nak);
        S->ckb[c] = scat(int64_t(c) << 4, t.bpk, t.nbk);
    }
    if (warp == kKdMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S->tmem)),
                     "r"(Sh::TmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = S->tmem;
    constexpr int mb = M == 16 ? 4 : 5, nb = N == 16 ? 4 : 5;

    if (warp < 4) {
        // ---------------- loaders: gather, split, store one K-chunk per stage ----------------
        // A row slot (key j, row m): 4 threads, 4 complex of the chunk each;
        // W column slot (key j, column n): 4 threads, 4 complex each.  The 4
        // threads of a slot are lanes 4i .. 4i + 3 of one warp and find the
        // slot's grid by shuffles.
        constexpr int kAS = NM * 4 / kKdLoadT;            // A slots per thread (NM rows x 4 quarters)
        constexpr int kWS = KPM * N * 4 / kKdLoadT;       // W slots per thread
        const int q4 = tid & 3;
        int64_t a_k[4], b_k[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            a_k[i] = scat(4 * q4 + i, t.apk, 4);
            b_k[i] = scat(4 * q4 + i, t.bpk, 4);
        }
        // chunk offsets of the summed index (bits >= 4 of k), one table per operand
        const int64_t* cka = S->cka;
        const int64_t* ckb = S->ckb;
        // Raw loads run RawDepth chunks ahead through cp.async into a ring in
        // shared memory; a thread later reads back exactly the values it
        // copied (element e of thread t at (e * 128 + t) * 8 bytes: a warp's
        // reads are one contiguous 256-byte run), so no barrier is needed.
        constexpr int R = Sh::RawDepth, PT = Sh::PerThread;
        float2* raw = reinterpret_cast<float2*>(sm + kStages * Sh::StageBytes);
        const int64_t total = (b_end - b_first) * nch;
        int64_t iblk = b_first - 1;
        int ic = nch;
        const float2* abi[kAS];
        const float2* bbi[kWS];
        auto issue = [&](int64_t idx) {
            if (idx < total) {
                if (ic == nch) {   // next key block: its operand bases
                    ic = 0;
                    ++iblk;
                    const int64_t u0 = iblk * KPM;
#pragma unroll
                    for (int s = 0; s < kAS; ++s) {
                        const int slot = (tid >> 2) + (kKdLoadT / 4) * s;   // row of the stacked A'^T
                        const int64_t u = u0 + slot / M;
                        abi[s] = u < t.kv ? arena + t.a_off + int64_t(t.uL[u]) * t.a_key + scat(slot % M, t.apm, mb)
                                          : nullptr;
                    }
#pragma unroll
                    for (int s = 0; s < kWS; ++s) {
                        const int slot = (tid >> 2) + (kKdLoadT / 4) * s;   // (key, column)
                        const int64_t u = u0 + slot / N;
                        bbi[s] = u < t.kv ? arena + t.b_off + int64_t(t.uR[u]) * t.b_key + scat(slot % N, t.bpn, nb)
                                          : nullptr;
                    }
                }
                float2* dst = raw + (idx % R) * (PT * 128) + tid;
#pragma unroll
                for (int s = 0; s < kAS; ++s)
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        cp_async8(dst + (s * 4 + i) * 128, abi[s] ? abi[s] + cka[ic] + a_k[i] : arena, abi[s] != nullptr);
#pragma unroll
                for (int s = 0; s < kWS; ++s)
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        cp_async8(dst + ((kAS + s) * 4 + i) * 128, bbi[s] ? bbi[s] + ckb[ic] + b_k[i] : arena,
                                  bbi[s] != nullptr);
                ++ic;
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        };
        for (int d = 0; d < R - 1; ++d) issue(d);
        bool ok = true;
        for (int64_t idx = 0; idx < total && ok; ++idx) {
            issue(idx + R - 1);
            asm volatile("cp.async.wait_group %0;" ::"n"(R - 1) : "memory");
            const float2* src = raw + (idx % R) * (PT * 128) + tid;
            float2 a[kAS][4], w[kWS][4];
#pragma unroll
            for (int s = 0; s < kAS; ++s)
#pragma unroll
                for (int i = 0; i < 4; ++i) a[s][i] = src[(s * 4 + i) * 128];
#pragma unroll
            for (int s = 0; s < kWS; ++s)
#pragma unroll
                for (int i = 0; i < 4; ++i) w[s][i] = src[((kAS + s) * 4 + i) * 128];
            const int st = int(idx % kStages);
            ok = __all_sync(0xffffffffu,
                            bar_wait(&S->empty[st], (uint32_t(idx / kStages) & 1) ^ 1, t.err, 41, t.wait_ns));
            if (!ok) break;
            unsigned char* wbp = sm + st * Sh::StageBytes;
            unsigned char* wsp = wbp + kWBytes;
            unsigned char* abp = wbp + 2 * kWBytes;
            unsigned char* asp = abp + Sh::ABytes;
#pragma unroll
            for (int s = 0; s < kAS; ++s) {
                const int row = (tid >> 2) + (kKdLoadT / 4) * s;
                float ma = 0.f;
#pragma unroll
                for (int i = 0; i < 4; ++i) ma = fmaxf(ma, fmaxf(fabsf(a[s][i].x), fabsf(a[s][i].y)));
                ma = fmaxf(ma, __shfl_xor_sync(0xffffffffu, ma, 1));
                ma = fmaxf(ma, __shfl_xor_sync(0xffffffffu, ma, 2));
                const float c0 = grid_c(ma, t.split_bits);
                float4 b, sm4;
                split4(make_float4(a[s][0].x, a[s][0].y, a[s][1].x, a[s][1].y), c0, b, sm4);
                *reinterpret_cast<float4*>(abp + kd_unit(row, 2 * q4)) = b;
                *reinterpret_cast<float4*>(asp + kd_unit(row, 2 * q4)) = sm4;
                split4(make_float4(a[s][2].x, a[s][2].y, a[s][3].x, a[s][3].y), c0, b, sm4);
                *reinterpret_cast<float4*>(abp + kd_unit(row, 2 * q4 + 1)) = b;
                *reinterpret_cast<float4*>(asp + kd_unit(row, 2 * q4 + 1)) = sm4;
            }
            // W^T rows 2 (N j + n) (real part of column n: Re B, -Im B per k) and
            // 2 (N j + n) + 1 (imaginary part: Im B, Re B)
#pragma unroll
            for (int s = 0; s < kWS; ++s) {
                const int slot = (tid >> 2) + (kKdLoadT / 4) * s;
                float mw = 0.f;
#pragma unroll
                for (int i = 0; i < 4; ++i) mw = fmaxf(mw, fmaxf(fabsf(w[s][i].x), fabsf(w[s][i].y)));
                mw = fmaxf(mw, __shfl_xor_sync(0xffffffffu, mw, 1));
                mw = fmaxf(mw, __shfl_xor_sync(0xffffffffu, mw, 2));
                const float cw = grid_c(mw, t.split_bits);
                const int r0 = 2 * slot, r1 = r0 + 1;
                const float2* x = w[s];
                float4 b, sm4;
                split4(make_float4(x[0].x, -x[0].y, x[1].x, -x[1].y), cw, b, sm4);
                *reinterpret_cast<float4*>(wbp + kd_unit(r0, 2 * q4)) = b;
                *reinterpret_cast<float4*>(wsp + kd_unit(r0, 2 * q4)) = sm4;
                split4(make_float4(x[2].x, -x[2].y, x[3].x, -x[3].y), cw, b, sm4);
                *reinterpret_cast<float4*>(wbp + kd_unit(r0, 2 * q4 + 1)) = b;
                *reinterpret_cast<float4*>(wsp + kd_unit(r0, 2 * q4 + 1)) = sm4;
                split4(make_float4(x[0].y, x[0].x, x[1].y, x[1].x), cw, b, sm4);
                *reinterpret_cast<float4*>(wbp + kd_unit(r1, 2 * q4)) = b;
                *reinterpret_cast<float4*>(wsp + kd_unit(r1, 2 * q4)) = sm4;
                split4(make_float4(x[2].y, x[2].x, x[3].y, x[3].x), cw, b, sm4);
                *reinterpret_cast<float4*>(wbp + kd_unit(r1, 2 * q4 + 1)) = b;
                *reinterpret_cast<float4*>(wsp + kd_unit(r1, 2 * q4 + 1)) = sm4;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            bar_arrive(&S->full[st]);
        }
        // no copy may be in flight when the CTA exits
        asm volatile("cp.async.wait_group 0;" ::: "memory");
    } else if (warp == kKdMmaWarp) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(NM >> 3) << 17) |
                                   (uint32_t(128 >> 4) << 24);
            const bool four = t.split_terms == 4;
            bool ok = true;
            // testing aid (xeb_plan_test_wait): a wait that runs out
            if (t.test_wait) ok = bar_wait(&S->never, 0, t.err, 30, t.wait_ns) && false;
            int64_t it = 0, sg = 0, q = 0;
            for (int64_t blk = b_first; blk < b_end && ok; ++blk, ++q) {
                const uint32_t dcr = tmem + 2 * NM + NM * uint32_t(q & 1);
                if (!bar_wait(&S->crempty[q & 1], (uint32_t(q >> 1) & 1) ^ 1, t.err, 42, t.wait_ns)) {
                    ok = false;
                    break;
                }
                fence_after();
                for (int c = 0; c < nch && ok; ++c, ++it) {
                    const uint32_t dbb = tmem + NM * uint32_t(sg & 1);
                    if (c % kSeg == 0) {
                        if (!bar_wait(&S->segempty[sg & 1], (uint32_t(sg >> 1) & 1) ^ 1, t.err, 43, t.wait_ns)) {
                            ok = false;
                            break;
                        }
                        fence_after();
                    }
                    const int st = int(it % kStages);
                    if (!bar_wait(&S->full[st], uint32_t(it / kStages) & 1, t.err, 44, t.wait_ns)) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    const uint32_t wb = smem_u32(sm + st * Sh::StageBytes), ws = wb + kWBytes, ab = wb + 2 * kWBytes,
                                   as = ab + Sh::ABytes;
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks) {
                        const uint32_t kb = ks * 32;
                        mma_ss(dbb, sdesc(wb + kb), sdesc(ab + kb), idesc, (c % kSeg != 0 || ks != 0) ? 1u : 0u);
                        mma_ss(dcr, sdesc(wb + kb), sdesc(as + kb), idesc, (c != 0 || ks != 0) ? 1u : 0u);
                        mma_ss(dcr, sdesc(ws + kb), sdesc(ab + kb), idesc, 1u);
                        if (four) mma_ss(dcr, sdesc(ws + kb), sdesc(as + kb), idesc, 1u);
                    }
                    mma_commit(&S->empty[st]);
                    if (c % kSeg == kSeg - 1) {
                        mma_commit(&S->segfull[sg & 1]);
                        ++sg;
                    }
                }
                if (!ok) break;
                mma_commit(&S->crfull[q & 1]);
            }
            mma_commit(&S->drain);
            bar_wait(&S->drain, 0, t.err, 45, t.wait_ns);
        }
        __syncwarp();
    } else {
        // ---------------- epilogue: sum the segments, add the cross terms, store ----------------
        const int qd = warp - kKdEpiWarp0;       // tensor-memory lane quarter
        const int r = 32 * qd + lane;            // W^T row of the stacked keys
        const int jkey = r / (2 * N), np = r % (2 * N), nn = np >> 1, cpart = np & 1;
        const int64_t c_n = scat(nn, t.cpn, nb);
        const uint32_t lanes = uint32_t(32 * qd) << 16;
        const uint32_t colj = uint32_t(M * jkey);   // D columns of this key
        int64_t sg = 0, q = 0;
        bool ok = true;
        for (int64_t blk = b_first; blk < b_end && ok; ++blk, ++q) {
            float acc[M];
#pragma unroll
            for (int i = 0; i < M; ++i) acc[i] = 0.f;
            for (int sgi = 0; sgi < nseg; ++sgi, ++sg) {
                ok = __all_sync(0xffffffffu, bar_wait(&S->segfull[sg & 1], uint32_t(sg >> 1) & 1, t.err, 46, t.wait_ns));
                if (!ok) break;
                fence_after();
                float v[M];
                tm_ldM<M>(tmem + lanes + NM * uint32_t(sg & 1) + colj, v);
                tm_wait_ld();
                fence_before();
                bar_arrive(&S->segempty[sg & 1]);
#pragma unroll
                for (int i = 0; i < M; ++i) acc[i] = __fadd_rn(acc[i], v[i]);
            }
            if (!ok) break;
            ok = __all_sync(0xffffffffu, bar_wait(&S->crfull[q & 1], uint32_t(q >> 1) & 1, t.err, 47, t.wait_ns));
            if (!ok) break;
            fence_after();
            float v[M];
            tm_ldM<M>(tmem + lanes + 2 * NM + NM * uint32_t(q & 1) + colj, v);
            tm_wait_ld();
            fence_before();
            bar_arrive(&S->crempty[q & 1]);
            const int64_t u = blk * KPM + jkey;
            if (u < t.kv) {
                float* C = reinterpret_cast<float*>(arena + t.c_off + u * t.c_key + c_n) + cpart;
#pragma unroll
                for (int i = 0; i < M; ++i) C[2 * S->cm[i]] = __fadd_rn(acc[i], v[i]);
            }
        }
    }
    fence_before();
    __syncthreads();
    if (warp == kKdMmaWarp) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Sh::TmemCols) : "memory");
    }
}

namespace {
template <int M, int N>
constexpr size_t kd_smem() {
    return 1024 + size_t(KdShape<M, N>::Stages) * KdShape<M, N>::StageBytes +
           size_t(KdShape<M, N>::RawDepth) * KdShape<M, N>::RawBytes + sizeof(SmKd);
}
static_assert(kd_smem<16, 16>() <= 232448 && kd_smem<32, 32>() <= 232448 && kd_smem<16, 32>() <= 232448 &&
                  kd_smem<32, 16>() <= 232448,
              "deep-K tensor-core contraction exceeds the shared memory of one CTA");

template <int M, int N>
cudaError_t prep_one() {
    return cudaFuncSetAttribute(k_tc_kdeep<M, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kd_smem<M, N>()));
}
template <int M, int N>
void launch_one(const KdDesc& d, float2* arena, int n_sms, cudaStream_t st) {
    const int64_t blocks = (d.kv + KdShape<M, N>::KPM - 1) / KdShape<M, N>::KPM;
    const int grid = int(blocks < n_sms ? blocks : n_sms);
    if (grid > 0) k_tc_kdeep<M, N><<<grid, kKdThreads, kd_smem<M, N>(), st>>>(d, arena);
}
}  // namespace

cudaError_t prepare_tc_kdeep() {
    cudaError_t e = prep_one<16, 16>();
    if (e == cudaSuccess) e = prep_one<32, 32>();
    if (e == cudaSuccess) e = prep_one<16, 32>();
    if (e == cudaSuccess) e = prep_one<32, 16>();
    return e;
}

cudaError_t launch_tc_kdeep(const KdDesc& d, float2* arena, int n_sms, cudaStream_t st) {
    if (d.M == 16 && d.N == 16) launch_one<16, 16>(d, arena, n_sms, st);
    else if (d.M == 32 && d.N == 32) launch_one<32, 32>(d, arena, n_sms, st);
    else if (d.M == 16 && d.N == 32) launch_one<16, 32>(d, arena, n_sms, st);
    else if (d.M == 32 && d.N == 16) launch_one<32, 16>(d, arena, n_sms, st);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace xebk
