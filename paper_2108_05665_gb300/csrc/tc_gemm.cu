// Split-precision complex contraction on the 5th-generation tensor cores
// (tcgen05, kind::tf32, accumulators in tensor memory).
//
// The pairwise contraction T*S of Eq. (elem-cont) with one key, C (M x N) =
// A (M x K) * B (K x N) in complex arithmetic, is computed as the real GEMM
//     C' (M x 2N) = A' (M x 2K) * W (2K x 2N),
// where A' is A's interleaved (re, im) storage read as floats and
//     W[2k][2n] = Re B, W[2k+1][2n] = -Im B, W[2k][2n+1] = Im B, W[2k+1][2n+1] = Re B,
// so C' is C's interleaved storage.  Every operand x is split as
// x ~ big + small with big = RN_tf32(x) and small = RN_tf32(x - big): both are
// exact TF32 values, so the tensor cores see them unchanged and the split
// error (~2^-22 |x|) is unbiased; C' = A'_big W_big + A'_big W_small +
// A'_small W_big accumulates in FP32 in tensor memory (small*small is below
// FP32 resolution).  The big*big term and the two cross terms go to separate
// accumulators that the epilogue adds in FP32 round-to-nearest.
//
// Roles (one CTA per SM, persistent over 128-row tiles):
//   warps 0-7  gather A rows through the per-leg address positions, split
//              them and store big/small into a shared-memory stage in the
//              128-byte-swizzled K-major layout the MMA reads; each thread
//              keeps the loads of the next two chunks in flight while it
//              converts the current one;
//   warp  12   allocates tensor memory and (one lane) issues the MMAs;
//   warps 8-11 move finished accumulators from tensor memory to global C.
// W (big and small) stays in shared memory for the whole kernel.  Every wait
// is bounded: after ~2 s a role records an error code, stops, and the CTA
// drains outstanding MMAs and frees its tensor memory before returning.
#include "kernels.cuh"

namespace xebk {

namespace {

constexpr int kTcRows = 128;       // rows per tile (UMMA M)
constexpr int kChunkFloats = 32;   // one 128-byte swizzle atom along K
constexpr int kStages = 2;
constexpr int kCStride = 33;       // staging row stride (floats): conflict-free both ways
constexpr int kLoaderWarps = 8;
constexpr int kLoaderThreads = 32 * kLoaderWarps;   // 256
                                                     // warps 8-11: epilogue
constexpr int kMmaWarp = kLoaderWarps + 4;           // warp 12: TMEM + MMA issue
constexpr int kThreads = 32 * (kLoaderWarps + 5);    // 416
constexpr int kElems = kTcRows * 16 / kLoaderThreads;  // A elements per loader thread per chunk (8)
constexpr uint64_t kWaitNs = 2000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return uint32_t(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Bounded wait; false (with *err set) on timeout or when another role failed.
__device__ bool mbar_wait(uint64_t* bar, uint32_t parity, int32_t* err, int code) {
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (uint32_t i = 0;; ++i) {
        if (mbar_try(bar, parity)) return true;
        if ((i & 255) == 255) {
            if (*reinterpret_cast<volatile int32_t*>(err) != 0) return false;
            if (globaltimer() - t0 > kWaitNs) {
                atomicCAS(err, 0, kErrTimeout | code);
                return false;
            }
        }
    }
}

// 128B-swizzle: 16-byte chunk index (address bits 4-6) XOR row-in-group (bits 7-9)
__device__ __forceinline__ uint32_t swz(uint32_t byte) { return byte ^ (((byte >> 7) & 7u) << 4); }

__device__ __forceinline__ float tf32_rn(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// K-major, 128-byte swizzled operand: rows of 128 B, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= uint64_t((saddr & 0x3FFFF) >> 4);
    d |= uint64_t(1) << 16;            // leading byte offset (unused for swizzled K-major)
    d |= uint64_t(1024 >> 4) << 32;    // stride byte offset between 8-row groups
    d |= uint64_t(1) << 46;            // descriptor version
    d |= uint64_t(2) << 61;            // SWIZZLE_128B
    return d;
}

__device__ __forceinline__ void umma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
        ::"r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

struct TcSmem {
    uint64_t full[kStages], empty[kStages], tfull[2], tempty[2], drain;
    uint32_t tmem_base;
};

}  // namespace

// W image (big then small): for chunk c, row n' (0..N2-1), 32 floats of K'
// at [c][n'] with the 128B swizzle, exactly as the MMA reads shared memory.
__global__ void k_tc_prep(const __grid_constant__ TcDesc t, const float2* __restrict__ arena) {
    const float2* B = arena + t.b_off;
    const int total = t.N2 * t.K2;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int np = e / t.K2, kp = e % t.K2;
        const int n = np >> 1, cpart = np & 1, k = kp >> 1, apart = kp & 1;
        int64_t off = 0;
        for (int i = 0; i < t.nbk; ++i)
            if ((k >> i) & 1) off |= int64_t(1) << t.bpk[i];
        for (int i = 0; i < t.nbn; ++i)
            if ((n >> i) & 1) off |= int64_t(1) << t.bpn[i];
        const float2 b = B[off];
        float w;
        if (cpart == 0) w = apart == 0 ? b.x : -b.y;
        else w = apart == 0 ? b.y : b.x;
        const float big = tf32_rn(w);
        const float small = tf32_rn(w - big);
        const int chunk = kp / kChunkFloats;
        const uint32_t byte = swz(uint32_t(np) * 128u + uint32_t(kp % kChunkFloats) * 4u);
        const int64_t idx = int64_t(chunk) * t.N2 * kChunkFloats + byte / 4;
        t.wimg[idx] = big;
        t.wimg[int64_t(t.n_chunks) * t.N2 * kChunkFloats + idx] = small;
    }
}

__global__ void __launch_bounds__(kThreads, 1) k_tc_gemm(const __grid_constant__ TcDesc t, float2* __restrict__ arena) {
    extern __shared__ __align__(1024) unsigned char sm_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(sm_raw) + 1023) & ~uintptr_t(1023));
    const int w_chunk_bytes = t.N2 * 128;                  // one K-chunk of W for all N2 rows
    const int w_bytes = t.n_chunks * w_chunk_bytes;        // big (small follows)
    float* Wbig = reinterpret_cast<float*>(sm);
    float* Wsmall = reinterpret_cast<float*>(sm + w_bytes);
    unsigned char* stage_base = sm + 2 * w_bytes;          // per stage: A big 16 KB, A small 16 KB
    const int stage_bytes = 2 * kTcRows * 128;
    float* Cstage = reinterpret_cast<float*>(stage_base + kStages * stage_bytes);  // 4 warps x 32 x 33
    TcSmem* S = reinterpret_cast<TcSmem*>(Cstage + 4 * 32 * kCStride);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t n_tiles = t.M / kTcRows;

    // W image -> shared memory (16-byte copies)
    {
        const int4* src = reinterpret_cast<const int4*>(t.wimg);
        int4* dst = reinterpret_cast<int4*>(sm);
        for (int i = tid; i < 2 * w_bytes / 16; i += kThreads) dst[i] = src[i];
    }
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&S->full[s], kLoaderThreads);
            mbar_init(&S->empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&S->tfull[b], 1);
            mbar_init(&S->tempty[b], 128);  // the 4 epilogue warps
        }
        mbar_init(&S->drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S->tmem_base)),
                     "r"(uint32_t(t.tmem_cols))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // W visible to the tensor cores
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S->tmem_base;

    if (warp < kLoaderWarps) {
        // ---------------- A producer: gather, split, swizzle ----------------
        // per-thread tile elements: e = tid + 256 j, tile bits (7 row bits +
        // 4 k bits of the chunk) in ascending address order
        int32_t off[kElems];
        uint32_t pos[kElems];
#pragma unroll
        for (int j = 0; j < kElems; ++j) {
            const int e = tid + kLoaderThreads * j;
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
        const int64_t total = my_tiles * t.n_chunks;
        auto issue = [&](int64_t it, float2 (&v)[kElems]) {
            if (it >= total) return;
            const int64_t tile = blockIdx.x + (it / t.n_chunks) * int64_t(gridDim.x);
            const int c = int(it % t.n_chunks);
            const int64_t m0 = tile * kTcRows;
            int64_t row_base = 0;
            for (int i = 7; i < t.nam; ++i)
                if ((m0 >> i) & 1) row_base |= int64_t(1) << t.apm[i];
            const float2* Ac = arena + t.a_off + row_base + t.chunk_off[c];
#pragma unroll
            for (int j = 0; j < kElems; ++j) v[j] = Ac[off[j]];
        };
        bool ok = true;
        auto store = [&](int64_t it, const float2 (&v)[kElems]) {
            if (!ok || it >= total) return;
            const int s = int(it % kStages);
            const uint32_t use = uint32_t(it / kStages);
            if (!mbar_wait(&S->empty[s], (use & 1) ^ 1, t.err, 1)) { ok = false; return; }
            unsigned char* sb = stage_base + s * stage_bytes;
#pragma unroll
            for (int j = 0; j < kElems; ++j) {
                const float bx = tf32_rn(v[j].x), by = tf32_rn(v[j].y);
                *reinterpret_cast<float2*>(sb + pos[j]) = make_float2(bx, by);
                *reinterpret_cast<float2*>(sb + kTcRows * 128 + pos[j]) =
                    make_float2(tf32_rn(v[j].x - bx), tf32_rn(v[j].y - by));
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(&S->full[s]);
        };
        float2 va[kElems], vb[kElems], vc[kElems];
        issue(0, va);
        issue(1, vb);
        for (int64_t it = 0; it < total && ok; it += 3) {
            issue(it + 2, vc);
            store(it, va);
            issue(it + 3, va);
            store(it + 1, vb);
            issue(it + 4, vb);
            store(it + 2, vc);
        }
    } else if (warp == kMmaWarp) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(t.N2 >> 3) << 17) |
                                   (uint32_t(kTcRows >> 4) << 24);
            const uint32_t wb = smem_u32(Wbig), ws = smem_u32(Wsmall);
            uint32_t it = 0, tcount = 0;
            bool ok = true;
            for (int64_t tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x, ++tcount) {
                const uint32_t b = tcount & 1, ub = tcount >> 1;
                if (!mbar_wait(&S->tempty[b], (ub & 1) ^ 1, t.err, 2)) break;
                tc_fence_after();
                // big*big in d_big; the two cross terms in d_small (the
                // tensor-core accumulation truncates, so tiny terms added to a
                // large accumulator would lose their low bits systematically)
                const uint32_t d_big = tmem + b * uint32_t(2 * t.N2);
                const uint32_t d_small = d_big + uint32_t(t.N2);
                for (int c = 0; c < t.n_chunks; ++c, ++it) {
                    const int s = int(it % kStages);
                    const uint32_t use = it / kStages;
                    if (!mbar_wait(&S->full[s], use & 1, t.err, 3)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t ab = smem_u32(stage_base + s * stage_bytes);
                    const uint32_t as = ab + kTcRows * 128;
                    const uint32_t wcb = wb + c * w_chunk_bytes, wcs = ws + c * w_chunk_bytes;
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks) {
                        const uint32_t kb = ks * 32;  // 8 tf32 along K
                        umma_tf32(d_big, umma_desc(ab + kb), umma_desc(wcb + kb), idesc, (c | ks) != 0);
                        umma_tf32(d_small, umma_desc(ab + kb), umma_desc(wcs + kb), idesc, (c | ks) != 0);
                        umma_tf32(d_small, umma_desc(as + kb), umma_desc(wcb + kb), idesc, 1);
                    }
                    umma_commit(&S->empty[s]);
                }
                if (!ok) break;
                umma_commit(&S->tfull[b]);
            }
            // every MMA issued by this thread has completed once drain fires
            umma_commit(&S->drain);
            mbar_wait(&S->drain, 0, t.err, 4);
        }
        __syncwarp();
    } else {
        // ---------------- epilogue: tensor memory -> C ----------------
        const int q = warp & 3;                 // lane quarter of this warp
        float* stg = Cstage + q * 32 * kCStride;
        uint32_t tcount = 0;
        for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++tcount) {
            const uint32_t b = tcount & 1, ub = tcount >> 1;
            const bool got = mbar_wait(&S->tfull[b], ub & 1, t.err, 5);
            if (!__all_sync(0xffffffffu, got)) break;
            tc_fence_after();
            // rows q*32 .. q*32+31 of this tile; each 32-column slice goes
            // through a padded staging buffer so that every warp store
            // writes four full 128-byte row segments
            float* Cw = reinterpret_cast<float*>(arena + t.c_off) + (tile * kTcRows + q * 32) * int64_t(t.N2);
            const uint32_t tb = tmem + (uint32_t(q * 32) << 16) + b * uint32_t(2 * t.N2);
            for (int c0 = 0; c0 < t.N2; c0 += 32) {
                float v[32], w[32];
                tmem_ld32(tb + uint32_t(c0), v);
                tmem_ld32(tb + uint32_t(t.N2 + c0), w);
#pragma unroll
                for (int i = 0; i < 32; ++i) stg[lane * kCStride + i] = v[i] + w[i];
                __syncwarp();
                const int rr = lane >> 3, cc = (lane & 7) * 4;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int row = rr + 4 * i;
                    const float* src = stg + row * kCStride + cc;
                    *reinterpret_cast<float4*>(Cw + int64_t(row) * t.N2 + c0 + cc) =
                        make_float4(src[0], src[1], src[2], src[3]);
                }
                __syncwarp();
            }
            tc_fence_before();
            mbar_arrive(&S->tempty[b]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == kMmaWarp) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(uint32_t(t.tmem_cols))
                     : "memory");
    }
}

size_t tc_wimg_floats(const TcDesc& t) { return size_t(2) * t.n_chunks * t.N2 * kChunkFloats; }

size_t tc_smem_bytes(const TcDesc& t) {
    const size_t w_bytes = size_t(t.n_chunks) * t.N2 * 128;
    return 1024 + 2 * w_bytes + size_t(kStages) * 2 * kTcRows * 128 + 4 * 32 * kCStride * 4 + sizeof(TcSmem);
}

cudaError_t prepare_tc1() {
    return cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
}

cudaError_t launch_tc_gemm(const TcDesc& t, float2* arena, int n_sms, cudaStream_t st) {
    k_tc_prep<<<64, 256, 0, st>>>(t, arena);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t tiles = t.M / kTcRows;
    const int grid = int(tiles < n_sms ? tiles : n_sms);
    k_tc_gemm<<<grid, kThreads, tc_smem_bytes(t), st>>>(t, arena);
    return cudaGetLastError();
}

}  // namespace xebk
