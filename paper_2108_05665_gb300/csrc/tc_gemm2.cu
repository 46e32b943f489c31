// Split-precision complex contraction on tcgen05 with the small operand in
// tensor memory.
//
// Same arithmetic as tc_gemm.cu (C' = A' W with the real expansion
// W = [[Re B, Im B], [-Im B, Re B]] interleaved, operands split into RN-TF32
// big + small, three products, big*big and the cross terms in separate FP32
// accumulators), with the roles of the MMA operands swapped:
//
//     D (2N x rows) = W^T (2N x 2K) * A'^T (2K x rows)
//
// W^T (big and small, <= 128 x 128 floats each) is written once per CTA into
// tensor memory and serves as the MMA's A operand; the state rows are the
// shared-memory B operand (K-major, 128-byte swizzle), so shared memory holds
// only a deep ring of state chunks.  The producer warps gather state elements
// with cp.async straight into the ring (the k legs of a contraction sit at
// arbitrary address bits), and split each chunk into big/small in place when
// its copies have landed.  One thread issues the MMAs; four epilogue warps
// read D^T from tensor memory (lane = output column), transpose it through a
// padded shared buffer and write whole rows of C.
//
// Tensor memory: columns [0, 128) W^T big, [128, 256) W^T small, [256, 384)
// big*big accumulator, [384, 512) cross-term accumulator (128-row tiles: one
// MMA instruction covers 128 state rows).  Every wait is
// bounded (2 s, error word); the CTA always drains its MMAs and frees tensor
// memory before returning.
#include "kernels.cuh"

namespace xebk {

namespace {

constexpr int kRows = 128;           // state rows per tile (UMMA N)
constexpr int kM = 128;              // W^T rows (UMMA M), N2 padded to 128
constexpr int kChunk = 32;           // floats of K' per chunk (one swizzle atom)
constexpr int kRing = 4;             // chunk stages (16 KB big + 16 KB small each)
constexpr int kProdWarps = 4;
constexpr int kProd = 32 * kProdWarps;            // 128 producer threads
constexpr int kEpiWarp0 = kProdWarps;             // warps 4-7
constexpr int kMmaWarp = kProdWarps + 4;          // warp 8
constexpr int kThreads = 32 * (kProdWarps + 5);   // 288
constexpr int kPerThread = kRows * 16 / kProd;    // 16 complex elements per producer per chunk
constexpr int kRowBits = 7;
constexpr int kTab = 256;                         // result-tile table entries
constexpr int kStageBytes = 2 * kRows * 128;      // big + small, 16 KB each
constexpr int kCStride = 132;                     // floats per staged output row
constexpr uint32_t kTmemCols = 512;
constexpr uint64_t kWaitNs = 2000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return uint32_t(__cvta_generic_to_shared(p)); }
__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void bar_init(uint64_t* b, uint32_t n) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void bar_arrive(uint64_t* b) {
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ bool bar_try(uint64_t* b, uint32_t par) {
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok)
                 : "r"(smem_u32(b)), "r"(par)
                 : "memory");
    return ok != 0;
}
__device__ bool bar_wait(uint64_t* b, uint32_t par, int32_t* err, int code) {
    if (bar_try(b, par)) return true;
    const uint64_t t0 = gtimer();
    for (uint32_t i = 0;; ++i) {
        if (bar_try(b, par)) return true;
        if ((i & 255) == 255) {
            if (*reinterpret_cast<volatile int32_t*>(err) != 0) return false;
            if (gtimer() - t0 > kWaitNs) {
                atomicCAS(err, 0, kErrTimeout | code);
                return false;
            }
        }
    }
}
__device__ __forceinline__ uint32_t swz(uint32_t byte) { return byte ^ (((byte >> 7) & 7u) << 4); }
__device__ __forceinline__ float tf32_rn(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    return uint64_t((saddr & 0x3FFFF) >> 4) | (uint64_t(1) << 16) | (uint64_t(1024 >> 4) << 32) |
           (uint64_t(1) << 46) | (uint64_t(2) << 61);
}
// D[tmem] (+)= A[tmem] * B[smem]
__device__ __forceinline__ void mma_ts(uint32_t d, uint32_t a_tmem, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}" ::"r"(d),
        "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* b) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(b))
                 : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void cp8(void* s, const void* g) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(s)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void tm_ld32(uint32_t ta, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(ta));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tm_st32(uint32_t ta, const float* v) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
        "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(ta),
        "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
        "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
        "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
        "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
        "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
        "r"(__float_as_uint(v[15])), "r"(__float_as_uint(v[16])), "r"(__float_as_uint(v[17])),
        "r"(__float_as_uint(v[18])), "r"(__float_as_uint(v[19])), "r"(__float_as_uint(v[20])),
        "r"(__float_as_uint(v[21])), "r"(__float_as_uint(v[22])), "r"(__float_as_uint(v[23])),
        "r"(__float_as_uint(v[24])), "r"(__float_as_uint(v[25])), "r"(__float_as_uint(v[26])),
        "r"(__float_as_uint(v[27])), "r"(__float_as_uint(v[28])), "r"(__float_as_uint(v[29])),
        "r"(__float_as_uint(v[30])), "r"(__float_as_uint(v[31]))
        : "memory");
}
struct Sm2 {
    uint64_t full[kRing], empty[kRing], tfull[2], tempty[2], wready, drain, epi;
    int64_t hi_glob[kTab];
    int32_t hi_slot[kTab];
    uint32_t tmem;
};

}  // namespace

__global__ void __launch_bounds__(kThreads, 1) k_tc_gemm2(const __grid_constant__ TcDesc t, float2* __restrict__ arena) {
    extern __shared__ __align__(1024) unsigned char raw2[];
    unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(raw2) + 1023) & ~uintptr_t(1023));
    unsigned char* ring = sm;                                         // kRing x (big 8 KB | small 8 KB)
    float* cst = reinterpret_cast<float*>(sm + kRing * kStageBytes);  // kRows x kCStride
    Sm2* S = reinterpret_cast<Sm2*>(cst + kRows * kCStride);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t n_tiles = t.M / kRows;
    const int nch = t.n_chunks;
    if (tid == 0) {
        for (int s = 0; s < kRing; ++s) {
            bar_init(&S->full[s], kProd);
            bar_init(&S->empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            bar_init(&S->tfull[b], 1);
            bar_init(&S->tempty[b], 128);
        }
        bar_init(&S->wready, 128);
        bar_init(&S->drain, 1);
        bar_init(&S->epi, 128);
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

    if (warp < kProdWarps) {
        // ---------------- producers: gather (cp.async) and split in place ----------------
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
        const int64_t my_tiles = n_tiles > blockIdx.x ? (n_tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
        const int64_t total = my_tiles * nch;
        constexpr int D = kRing - 2;   // chunks whose copies are in flight ahead of the split
        bool ok = true;
        int64_t tile_of = -1, base = 0;
        int c = 0;
        int64_t tcur = blockIdx.x;
        for (int64_t it = 0; it < total + D && ok; ++it) {
            if (it < total) {
                const int s = int(it % kRing);
                const uint32_t use = uint32_t(it / kRing);
                if (!bar_wait(&S->empty[s], (use & 1) ^ 1, t.err, 11)) { ok = false; break; }
                if (tile_of != tcur) {
                    tile_of = tcur;
                    base = 0;
                    for (int i = 0; i < t.n_ext; ++i)
                        if ((tcur >> i) & 1) base |= int64_t(1) << t.ext_apos[i];
                }
                const float2* A = arena + t.a_off + base + t.chunk_off[c];
                unsigned char* sb = ring + s * kStageBytes;
#pragma unroll
                for (int j = 0; j < kPerThread; ++j) cp8(sb + pos[j], A + off[j]);
                if (++c == nch) { c = 0; tcur += gridDim.x; }
            }
            cp_commit();
            if (it >= D) {
                // copies of chunk it-D have landed: split big/small in place
                cp_wait<D>();
                const int64_t jt = it - D;
                const int s = int(jt % kRing);
                unsigned char* sb = ring + s * kStageBytes;
#pragma unroll
                for (int j = 0; j < kPerThread; ++j) {
                    float2* pb = reinterpret_cast<float2*>(sb + pos[j]);
                    const float2 v = *pb;
                    const float bx = tf32_rn(v.x), by = tf32_rn(v.y);
                    *pb = make_float2(bx, by);
                    *reinterpret_cast<float2*>(sb + kRows * 128 + pos[j]) =
                        make_float2(tf32_rn(v.x - bx), tf32_rn(v.y - by));
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                bar_arrive(&S->full[s]);
            }
        }
        cp_wait<0>();
    } else if (warp == kMmaWarp) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(kRows >> 3) << 17) |
                                   (uint32_t(kM >> 4) << 24);
            bool ok = bar_wait(&S->wready, 0, t.err, 12);
            fence_after();
            uint32_t it = 0, tc = 0;
            for (int64_t tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x, ++tc) {
                const uint32_t b = 0, ub = tc;  // one accumulator pair (TMEM is full)
                if (!bar_wait(&S->tempty[b], (ub & 1) ^ 1, t.err, 13)) break;
                fence_after();
                const uint32_t d_big = tmem + 256, d_small = d_big + kRows;
                for (int ch = 0; ch < nch; ++ch, ++it) {
                    const int s = int(it % kRing);
                    const uint32_t use = it / kRing;
                    if (!bar_wait(&S->full[s], use & 1, t.err, 14)) { ok = false; break; }
                    fence_after();
                    const uint32_t sb = smem_u32(ring + s * kStageBytes), ss = sb + kRows * 128;
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks) {
                        const uint32_t kc = uint32_t(ch * kChunk + ks * 8);  // TMEM column of this K step
                        const uint32_t kb = ks * 32;                          // byte offset in the swizzle atom
                        mma_ts(d_big, w_big + kc, sdesc(sb + kb), idesc, (ch | ks) != 0);
                        mma_ts(d_small, w_small + kc, sdesc(sb + kb), idesc, (ch | ks) != 0);
                        mma_ts(d_small, w_big + kc, sdesc(ss + kb), idesc, 1);
                    }
                    mma_commit(&S->empty[s]);
                }
                if (!ok) break;
                mma_commit(&S->tfull[b]);
            }
            mma_commit(&S->drain);
            bar_wait(&S->drain, 0, t.err, 15);
        }
        __syncwarp();
    } else {
        // ---------------- W^T into tensor memory, then the epilogue ----------------
        const int q = warp - kEpiWarp0;          // lane quarter (warps 4..7 -> 0..3)
        const int np = q * 32 + lane;            // W^T row = output column n' (0..127)
        {
            const int n = np >> 1, cpart = np & 1;
            const bool live = np < t.N2;
            int64_t noff = 0;
            if (live)
                for (int i = 0; i < t.nbn; ++i)
                    if ((n >> i) & 1) noff |= int64_t(1) << t.bpn[i];
            const float2* B = arena + t.b_off;
            for (int c0 = 0; c0 < t.K2; c0 += 32) {
                float vb[32], vs[32];
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const int kp = c0 + i, k = kp >> 1, apart = kp & 1;
                    float w = 0.f;
                    if (live) {
                        int64_t off = noff;
                        for (int b = 0; b < t.nbk; ++b)
                            if ((k >> b) & 1) off |= int64_t(1) << t.bpk[b];
                        const float2 bv = B[off];
                        w = cpart == 0 ? (apart == 0 ? bv.x : -bv.y) : (apart == 0 ? bv.y : bv.x);
                    }
                    vb[i] = tf32_rn(w);
                    vs[i] = tf32_rn(w - vb[i]);
                }
                const uint32_t lanes = uint32_t(q * 32) << 16;
                tm_st32(w_big + lanes + uint32_t(c0), vb);
                tm_st32(w_small + lanes + uint32_t(c0), vs);
            }
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            fence_before();
            bar_arrive(&S->wready);
        }
        uint32_t tc = 0, ep = 0;
        const uint32_t lanes = uint32_t(q * 32) << 16;
        const int etid = tid - 32 * kEpiWarp0;   // 0..127
        // result tile element e (bits in ascending C address) -> staging slot
        // and C offset; split as e = e_hi * 32 + lane: the lane part once per
        // thread, the e_hi part in a per-CTA table
        int lo_slot = 0;
        int64_t lo_glob = 0;
        {
            int r = 0, n = 0;
            for (int i = 0; i < 5 && i < t.Tst; ++i) {
                const int bit = (lane >> i) & 1;
                if (!bit) continue;
                if ((t.st_is_n >> i) & 1) n |= 1 << t.st_idx[i];
                else r |= 1 << t.st_idx[i];
                lo_glob |= int64_t(1) << t.st_pos[i];
            }
            lo_slot = r * (kCStride / 2) + n;
        }
        const int n_hi = t.Tst > 5 ? 1 << (t.Tst - 5) : 1;
        for (int h = etid; h < n_hi; h += 128) {  // n_hi <= kTab
            int r = 0, n = 0;
            int64_t g = 0;
            for (int i = 5; i < t.Tst; ++i) {
                if (!((h >> (i - 5)) & 1)) continue;
                if ((t.st_is_n >> i) & 1) n |= 1 << t.st_idx[i];
                else r |= 1 << t.st_idx[i];
                g |= int64_t(1) << t.st_pos[i];
            }
            S->hi_slot[h] = r * (kCStride / 2) + n;
            S->hi_glob[h] = g;
        }
        // bounded sync of the four epilogue warps (an aborting warp cannot
        // leave the others blocked)
        auto epi_sync = [&]() {
            bar_arrive(&S->epi);
            const bool ok = bar_wait(&S->epi, ep & 1, t.err, 17);
            ++ep;
            return ok;
        };
        bool table_ok = __all_sync(0xffffffffu, epi_sync());  // table visible to all four warps
        for (int64_t tile = blockIdx.x; tile < n_tiles && table_ok; tile += gridDim.x, ++tc) {
            const uint32_t b = 0, ub = tc;
            const bool got = bar_wait(&S->tfull[b], ub & 1, t.err, 16);
            if (!__all_sync(0xffffffffu, got)) break;
            fence_after();
            // D^T: lane = output column np, column = tile row
            const uint32_t db = tmem + 256;
            for (int r0 = 0; r0 < kRows; r0 += 32) {
                float v[32], w[32];
                tm_ld32(db + lanes + uint32_t(r0), v);
                tm_ld32(db + lanes + kRows + uint32_t(r0), w);
#pragma unroll
                for (int i = 0; i < 32; ++i) cst[(r0 + i) * kCStride + np] = v[i] + w[i];
            }
            fence_before();
            bar_arrive(&S->tempty[b]);
            if (!__all_sync(0xffffffffu, epi_sync())) break;
            // the tile's results in ascending C address order (contiguous runs)
            int64_t cbase = 0;
            for (int i = 0; i < t.n_ext; ++i)
                if ((tile >> i) & 1) cbase |= int64_t(1) << t.ext_cpos[i];
            float2* C = arena + t.c_off + cbase + lo_glob;
            const float2* st2 = reinterpret_cast<const float2*>(cst);
            for (int h = q; h < n_hi; h += 4) C[S->hi_glob[h]] = st2[S->hi_slot[h] + lo_slot];
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

// 1024 bytes of alignment slack + ring + output staging + barriers/tables
size_t tc2_smem_bytes() {
    return 1024 + size_t(kRing) * kStageBytes + size_t(kRows) * kCStride * 4 + sizeof(Sm2);
}
static_assert(sizeof(Sm2) % 8 == 0 && 1024 + kRing * kStageBytes + kRows * kCStride * 4 + sizeof(Sm2) <= 232448,
              "tensor-memory contraction exceeds the shared memory of one CTA");

cudaError_t prepare_tc1();

cudaError_t prepare_tc_kernels() {
    cudaError_t e = prepare_tc1();
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_tc_gemm2, cudaFuncAttributeMaxDynamicSharedMemorySize, int(tc2_smem_bytes()));
}

cudaError_t launch_tc_gemm2(const TcDesc& t, float2* arena, int n_sms, cudaStream_t st) {
    const int64_t tiles = t.M / kRows;
    const int grid = int(tiles < n_sms ? tiles : n_sms);
    k_tc_gemm2<<<grid, kThreads, tc2_smem_bytes(), st>>>(t, arena);
    return cudaGetLastError();
}

}  // namespace xebk
