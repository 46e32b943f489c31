// Inline-PTX helpers of the tcgen05 split-precision kernels (tc_gemm2.cu,
// tc_kdeep.cu): mbarriers with bounded waits, TMA loads, shared-memory
// operand descriptors, MMA issue and commit, tensor-memory loads and stores,
// and the common-grid split of FP32 values into a TF32 big part and a TF32
// small part.
#pragma once

#include "kernels.cuh"

namespace xebk {
namespace {

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
// bounded wait: gives up (false) when the error word is set or after lim ns,
// recording kErrTimeout | code
__device__ bool bar_wait(uint64_t* b, uint32_t par, int32_t* err, int code, uint64_t lim) {
    if (bar_try(b, par)) return true;
    const uint64_t t0 = gtimer();
    for (uint32_t i = 0;; ++i) {
        if (bar_try(b, par)) return true;
        if ((i & 255) == 255) {
            if (*reinterpret_cast<volatile int32_t*>(err) != 0) return false;
            if (gtimer() - t0 > lim) {
                atomicCAS(err, 0, kErrTimeout | code);
                return false;
            }
        }
    }
}
// bounded wait that ignores the error word (waiting for copies in flight)
__device__ void bar_wait_drain(uint64_t* b, uint32_t par, uint64_t lim) {
    const uint64_t t0 = gtimer();
    for (uint32_t i = 0;; ++i) {
        if (bar_try(b, par)) return;
        if ((i & 255) == 255 && gtimer() - t0 > lim) return;
    }
}
__device__ __forceinline__ void bar_expect_tx(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
// 3-D tiled TMA load (x = floats of a chunk, y = rows, z = chunks) completing
// on mbarrier b
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* b) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(b))
        : "memory");
}
__device__ __forceinline__ uint32_t swz(uint32_t byte) { return byte ^ (((byte >> 7) & 7u) << 4); }
__device__ __forceinline__ float tf32_rn(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}
// Common-grid split (see the top of tc_gemm2.cu).  grid_c(m, bits) is the
// constant c = 1.5 * 2^(e - bits + 24) for a group whose largest magnitude m
// lies in [2^e, 2^(e+1)): for |x| <= m, (x + c) - c rounds x to the nearest
// multiple of u = 2^(e - bits + 1) (ties to even), because x + c stays in the
// binade of c whose spacing is u; the subtraction is exact.  m = 0 or a
// subnormal m takes e = -126.
__device__ __forceinline__ float grid_c(float m, int bits) {
    int ex = int((__float_as_uint(m) >> 23) & 0xffu);   // biased exponent of m (m >= 0)
    ex = ex < 1 ? 1 : ex;
    int cex = ex + 24 - bits;                            // biased exponent of c
    cex = cex > 254 ? 254 : cex;
    return __uint_as_float((uint32_t(cex) << 23) | 0x400000u);
}
__device__ __forceinline__ float grid_big(float x, float c) { return __fsub_rn(__fadd_rn(x, c), c); }
// big and small parts of x on the grid of c
__device__ __forceinline__ void split_on(float x, float c, float& big, float& small) {
    big = grid_big(x, c);
    small = tf32_rn(__fsub_rn(x, big));
}
__device__ __forceinline__ float absmax4(float4 v) {
    return fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w)));
}
__device__ __forceinline__ void split4(float4 v, float c, float4& b, float4& s) {
    split_on(v.x, c, b.x, s.x);
    split_on(v.y, c, b.y, s.y);
    split_on(v.z, c, b.z, s.z);
    split_on(v.w, c, b.w, s.w);
}
// shared-memory operand descriptor: K-major, 128-byte swizzle, 8-row groups
// sbo bytes apart (1024 when the groups are contiguous)
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t sbo = 1024) {
    return uint64_t((saddr & 0x3FFFF) >> 4) | (uint64_t(1) << 16) | (uint64_t(sbo >> 4) << 32) |
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
// D[tmem] (+)= A[smem] * B[smem]
__device__ __forceinline__ void mma_ss(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* b) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(b))
                 : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// 32 lanes x 32 columns of tensor memory into registers (no wait)
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
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
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
__device__ __forceinline__ void tm_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
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

}  // namespace
}  // namespace xebk
