// Keyed contractions with a deep summed index on tcgen05 (split precision).
//
// C_u = A_uL(u) (M x K) * B_uR(u) (K x N) for every key u of a keyed
// contraction (App. A: 2^(q+r) multiply-adds per key), (M, N) in {(16, 16),
// (32, 32), (16, 32)} complex ((32, 16) runs as the transposed product
// C_u^T = B^T A^T), K a multiple of 64 complex.  These are the contractions
// near the root of sliced plans: each key owns a small result and sums
// thousands of terms.
//
// Real expansion and split as in tc_gemm2.cu: per key D (2N x M) = W^T (2N x
// 2K) * A'^T (2K x M), W = [[Re B, Im B], [-Im B, Re B]] interleaved; every
// value is split into a TF32 big part on a common grid (one grid per row of a
// 32-float K-chunk: a row of A', a row of W^T) and a TF32 small part; big*big
// and big*small + small*big + small*small go to separate FP32 accumulators.
//
// Keys are stacked block-diagonally: KPM = 128 / (2N) keys per MMA.  W^T of
// key j fills tensor-memory lanes 2N j .. 2N (j + 1) - 1 (the MMA's A
// operand, M = 128) and A'^T of key j rows M j .. M (j + 1) - 1 of an NM = KPM
// M row shared-memory operand (the MMA's B operand, N = NM), so one MMA (K =
// 8) computes every key's product in the diagonal blocks of D (the rest of D
// is never read).  A stage holds one K-chunk of 16 complex (32 floats): W^T
// big and small in 2 x 32 tensor-memory columns, A'^T big and small in shared
// memory (one 128-byte swizzle line per row).  The MMAs read only the NM-row
// operand from shared memory, and the raw values go from global memory
// straight to registers.
//
// Exactness of the big*big sums needs them to stay below 2^24 grid units, so
// the big*big chain restarts every 4 chunks (K' = 128) in one of two
// tensor-memory accumulators (ping-pong); the epilogue adds each finished
// segment to FP32 registers with round-to-nearest while the MMAs run on into
// the other one.  The cross terms use one accumulator per key block (two,
// ping-pong across blocks).
//
// Warps: 0-7 load and split, two sets of four taking alternate chunks (warp w
// writes tensor-memory lanes 32 (w mod 4) .. 32 (w mod 4) + 31, the W^T rows
// it owns); 8-11 are the epilogue (warp 8 + q reads lanes 32q .. 32q + 31);
// warp 12 issues the MMAs.  Every wait is bounded (opts.timeout_ms, error
// word); the CTA drains its MMAs and frees tensor memory before it returns.
#include "kernels.cuh"
#include "tc_common.cuh"

namespace xebk {

namespace {

constexpr int kKdLoadWarps = 8;
constexpr int kKdSetT = 128;        // threads of one loader set
constexpr int kKdEpiWarp0 = 8;
constexpr int kKdMmaWarp = 12;
constexpr int kKdThreads = 32 * 13;
constexpr int kSeg = 4;             // chunks per big*big segment (K' = 128)
constexpr int kKdStages = 4;        // two per loader set
constexpr uint32_t kKdTmemCols = 512;

template <int M, int N>
struct KdShape {
    static constexpr int KPM = 128 / (2 * N);   // keys per MMA
    static constexpr int NM = KPM * M;          // A'^T rows = MMA N
    static constexpr int ABytes = NM * 128;     // one part (big or small) of A'^T per chunk
    static constexpr int StageBytes = 2 * ABytes;
    static constexpr int TPR = kKdSetT / NM;    // loader threads per A'^T row
    static constexpr int CPT = 16 / TPR;        // complex of that row per thread
    static constexpr uint32_t WCol0 = 4 * NM;   // W^T stages after the four accumulators
    static_assert(NM == 32 || NM == 64, "stacked keys: MMA N of 32 or 64");
    static_assert(WCol0 + 64 * kKdStages <= kKdTmemCols, "tensor memory of the stacked keys");
};

constexpr int kMaxChunks = 512;     // K <= 8192 complex
struct SmKd {
    uint64_t full[kKdStages], empty[kKdStages], segfull[2], segempty[2], crfull[2], crempty[2], drain, never;
    uint32_t tmem, pad;
    int64_t cm[32];                 // C offset of result row m
    int64_t cka[kMaxChunks], ckb[kMaxChunks];   // A / B offset of K-chunk c (k bits >= 4)
    int64_t ako[8], bko[8];         // A / B offset of k = 0 .. 7 inside a chunk (k bits 0-2)
};

__device__ __forceinline__ int64_t scat(int64_t x, const int8_t* pos, int n) {
    int64_t o = 0;
    for (int i = 0; i < n; ++i)
        if ((x >> i) & 1) o |= int64_t(1) << pos[i];
    return o;
}

// swizzled byte offset of 16-byte unit u of 128-byte row r (1024-byte atoms)
__device__ __forceinline__ uint32_t kd_unit(int r, int u) { return uint32_t(r * 128 + ((u ^ (r & 7)) << 4)); }

// registers into 32 lanes x 16 columns of tensor memory (no wait)
__device__ __forceinline__ void tm_st16(uint32_t ta, const float* v) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
            ta),
        "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
        "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
        "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
        "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
        "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
        "r"(__float_as_uint(v[15]))
        : "memory");
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
    constexpr int KPM = Sh::KPM, NM = Sh::NM, TPR = Sh::TPR, CPT = Sh::CPT;
    extern __shared__ __align__(1024) unsigned char kd_raw[];
    unsigned char* sm = kd_raw + ((1024u - (smem_u32(kd_raw) & 1023u)) & 1023u);
    SmKd* S = reinterpret_cast<SmKd*>(sm + kKdStages * Sh::StageBytes);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nch = t.K / 16;               // K-chunks per key
    const int nseg = nch / kSeg;
    // this CTA's key blocks (KPM consecutive keys each)
    const int64_t n_blocks = (t.kv + KPM - 1) / KPM;
    const int64_t per = (n_blocks + gridDim.x - 1) / gridDim.x;
    const int64_t b_first = int64_t(blockIdx.x) * per;
    const int64_t b_end = b_first + per < n_blocks ? b_first + per : n_blocks;
    if (tid == 0) {
        for (int s = 0; s < kKdStages; ++s) {
            bar_init(&S->full[s], kKdSetT);
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
    if (tid < 8) {
        S->ako[tid] = scat(tid, t.apk, 3);
        S->bko[tid] = scat(tid, t.bpk, 3);
    }
    if (warp == kKdMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S->tmem)),
                     "r"(kKdTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = S->tmem;
    constexpr int mb = M == 16 ? 4 : 5, nb = N == 16 ? 4 : 5;

    if (warp < kKdLoadWarps) {
        // ---------------- loaders: gather, split, store one K-chunk per stage ----------------
        // Set s (warps 4s .. 4s + 3) takes chunks s, s + 2, ... of the CTA's
        // sequence and so stages s, s + 2.  Thread (q, lane) of a set owns W^T
        // row r = 32 q + lane (tensor-memory lane r: the Re (r even) or Im (r
        // odd) part of column n of key j) and one TPR-th of A'^T row ra (CPT
        // complex).  The two threads of a W^T column each load 8 of its 16
        // complex and swap them by a shuffle; the TPR threads of an A'^T row
        // are adjacent lanes and find the row's grid by shuffles.
        const int set = warp >> 2, q = warp & 3, ltid = tid & (kKdSetT - 1);
        const int r = 32 * q + lane;
        const int slot = r >> 1, cpart = r & 1;
        const int jw = slot / N;
        const int64_t w_n = scat(slot % N, t.bpn, nb) + (cpart ? int64_t(1) << t.bpk[3] : 0);
        const int ra = ltid / TPR, pa = ltid % TPR;
        const int ja = ra / M;
        // k = pa * CPT + i: bit 3 of k is pa's when CPT = 8, bits 2-3 when CPT = 4
        int64_t a_m = scat(ra % M, t.apm, mb);
        if constexpr (CPT == 8) {
            if (pa & 1) a_m += int64_t(1) << t.apk[3];
        } else {
            if (pa & 1) a_m += int64_t(1) << t.apk[2];
            if (pa & 2) a_m += int64_t(1) << t.apk[3];
        }
        const uint32_t lanes = uint32_t(32 * q) << 16;
        const int64_t total = (b_end - b_first) * nch;
        int64_t base_blk = -1;
        const float2* wbase = nullptr;
        const float2* abase = nullptr;
        // raw values of chunk idx into registers (zeros past the last key)
        auto fetch = [&](int64_t idx, float2* w, float2* a) {
            if (idx >= total) return;
            const int64_t bi = idx / nch;
            const int c = int(idx - bi * nch);
            const int64_t blk = b_first + bi;
            if (blk != base_blk) {
                base_blk = blk;
                const int64_t uw = blk * KPM + jw, ua = blk * KPM + ja;
                wbase = uw < t.kv ? arena + t.b_off + int64_t(t.uR[uw]) * t.b_key + w_n : nullptr;
                abase = ua < t.kv ? arena + t.a_off + int64_t(t.uL[ua]) * t.a_key + a_m : nullptr;
            }
            if (wbase) {
                const float2* p = wbase + S->ckb[c];
#pragma unroll
                for (int i = 0; i < 8; ++i) w[i] = __ldg(p + S->bko[i]);
            } else {
#pragma unroll
                for (int i = 0; i < 8; ++i) w[i] = make_float2(0.f, 0.f);
            }
            if (abase) {
                const float2* p = abase + S->cka[c];
#pragma unroll
                for (int i = 0; i < CPT; ++i) a[i] = __ldg(p + S->ako[i]);
            } else {
#pragma unroll
                for (int i = 0; i < CPT; ++i) a[i] = make_float2(0.f, 0.f);
            }
        };
        float2 w[8], a[CPT];
        fetch(set, w, a);
        for (int64_t idx = set; idx < total; idx += 2) {
            float2 wn[8], an[CPT];
            fetch(idx + 2, wn, an);
            const int st = int(idx % kKdStages);
            const bool ok = __all_sync(
                0xffffffffu, bar_wait(&S->empty[st], (uint32_t(idx / kKdStages) & 1) ^ 1, t.err, 41, t.wait_ns));
            if (!ok) break;
            fence_after();
            // W^T row r: (Re B, -Im B) per k for the real part of column n,
            // (Im B, Re B) for the imaginary part; complex 8h .. 8h + 7 of the
            // chunk are this thread's w for h = cpart, its partner's otherwise
            float mw = 0.f;
#pragma unroll
            for (int i = 0; i < 8; ++i) mw = fmaxf(mw, fmaxf(fabsf(w[i].x), fabsf(w[i].y)));
            mw = fmaxf(mw, __shfl_xor_sync(0xffffffffu, mw, 1));
            const float cw = grid_c(mw, t.split_bits);
            const uint32_t wcol = tmem + lanes + Sh::WCol0 + 64u * uint32_t(st);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                float vb[16], vs[16];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const float ox = __shfl_xor_sync(0xffffffffu, w[i].x, 1);
                    const float oy = __shfl_xor_sync(0xffffffffu, w[i].y, 1);
                    const bool own = h == cpart;
                    const float xr = own ? w[i].x : ox, xi = own ? w[i].y : oy;
                    split_on(cpart ? xi : xr, cw, vb[2 * i], vs[2 * i]);
                    split_on(cpart ? xr : -xi, cw, vb[2 * i + 1], vs[2 * i + 1]);
                }
                tm_st16(wcol + 16u * h, vb);
                tm_st16(wcol + 32u + 16u * h, vs);
            }
            // A'^T row ra: (Re A, Im A) per k
            float ma = 0.f;
#pragma unroll
            for (int i = 0; i < CPT; ++i) ma = fmaxf(ma, fmaxf(fabsf(a[i].x), fabsf(a[i].y)));
#pragma unroll
            for (int o = 1; o < TPR; o <<= 1) ma = fmaxf(ma, __shfl_xor_sync(0xffffffffu, ma, o));
            const float ca = grid_c(ma, t.split_bits);
            unsigned char* abp = sm + st * Sh::StageBytes;
            unsigned char* asp = abp + Sh::ABytes;
#pragma unroll
            for (int v = 0; v < CPT / 2; ++v) {
                float4 b, s4;
                split4(make_float4(a[2 * v].x, a[2 * v].y, a[2 * v + 1].x, a[2 * v + 1].y), ca, b, s4);
                const int unit = pa * (CPT / 2) + v;
                *reinterpret_cast<float4*>(abp + kd_unit(ra, unit)) = b;
                *reinterpret_cast<float4*>(asp + kd_unit(ra, unit)) = s4;
            }
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            fence_before();
            bar_arrive(&S->full[st]);
#pragma unroll
            for (int i = 0; i < 8; ++i) w[i] = wn[i];
#pragma unroll
            for (int i = 0; i < CPT; ++i) a[i] = an[i];
        }
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
                    const int st = int(it % kKdStages);
                    if (!bar_wait(&S->full[st], uint32_t(it / kKdStages) & 1, t.err, 44, t.wait_ns)) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    const uint32_t wb = tmem + Sh::WCol0 + 64u * uint32_t(st), ws = wb + 32u;
                    const uint32_t ab = smem_u32(sm + st * Sh::StageBytes), as = ab + Sh::ABytes;
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks) {
                        const uint32_t kc = 8u * ks, kb = 32u * ks;
                        mma_ts(dbb, wb + kc, sdesc(ab + kb), idesc, (c % kSeg != 0 || ks != 0) ? 1u : 0u);
                        mma_ts(dcr, wb + kc, sdesc(as + kb), idesc, (c != 0 || ks != 0) ? 1u : 0u);
                        mma_ts(dcr, ws + kc, sdesc(ab + kb), idesc, 1u);
                        if (four) mma_ts(dcr, ws + kc, sdesc(as + kb), idesc, 1u);
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
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kKdTmemCols) : "memory");
    }
}

namespace {
template <int M, int N>
constexpr size_t kd_smem() {
    return 1024 + size_t(kKdStages) * KdShape<M, N>::StageBytes + sizeof(SmKd);
}
static_assert(kd_smem<16, 16>() <= 232448 && kd_smem<32, 32>() <= 232448 && kd_smem<16, 32>() <= 232448,
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

// C_u^T = B_uR(u)^T A_uL(u)^T: the roles of the two operands and of the
// result's row and column bits exchanged
KdDesc transposed(const KdDesc& d) {
    KdDesc e = d;
    e.a_off = d.b_off;
    e.a_key = d.b_key;
    e.b_off = d.a_off;
    e.b_key = d.a_key;
    e.uL = d.uR;
    e.uR = d.uL;
    e.M = d.N;
    e.N = d.M;
    e.nak = d.nbk;
    e.nbk = d.nak;
    for (int i = 0; i < 5; ++i) {
        e.apm[i] = d.bpn[i];
        e.bpn[i] = d.apm[i];
        e.cpm[i] = d.cpn[i];
        e.cpn[i] = d.cpm[i];
    }
    for (int i = 0; i < kMaxLegs; ++i) {
        e.apk[i] = d.bpk[i];
        e.bpk[i] = d.apk[i];
    }
    return e;
}
}  // namespace

cudaError_t prepare_tc_kdeep() {
    cudaError_t e = prep_one<16, 16>();
    if (e == cudaSuccess) e = prep_one<32, 32>();
    if (e == cudaSuccess) e = prep_one<16, 32>();
    return e;
}

cudaError_t launch_tc_kdeep(const KdDesc& d, float2* arena, int n_sms, cudaStream_t st) {
    if (d.M == 16 && d.N == 16) launch_one<16, 16>(d, arena, n_sms, st);
    else if (d.M == 32 && d.N == 32) launch_one<32, 32>(d, arena, n_sms, st);
    else if (d.M == 16 && d.N == 32) launch_one<16, 32>(d, arena, n_sms, st);
    else if (d.M == 32 && d.N == 16) launch_one<16, 32>(transposed(d), arena, n_sms, st);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace xebk
