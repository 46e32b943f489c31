// Keyed contractions with few summed values and narrow results (SIMT, FP32).
//
// C_u (M x N) = A_uL(u) (M x K) * B_uR(u) (K x N) for every key u of a keyed
// contraction (Eq. of the pairwise contraction evaluated once per memo key,
// App. A), K in {4, 8, 16, 32}, N in {1, 2, 4, 8, 16} complex, results
// row-major [M][N] per key.  Keys are ordered by left key, so the keys of a
// group (gstart[g] .. gstart[g + 1] - 1) share one A.  These contractions
// (the memo-trie levels, N = 1, and the wide keyed contractions of sliced
// plans) move M K complex of A per group and write M N per key: they are
// bound by memory and by the FP32 multiply-adds (4 K per output).
//
// One warp takes 32 consecutive rows of one group (a work item), lane = row:
// the lane holds its row's K values of A in registers (loaded one item ahead)
// and walks the group's keys, reading each key's B as uniform 16-byte loads
// (the same address in every lane: one L1 transaction) from a packed copy of
// the kvB distinct right operands (k_keyed_pack_b: [ub][k][n] contiguous).  A
// warp's results for one key are 32 consecutive rows of N complex: one
// contiguous run.  N = 1 takes two keys per pass so that every 16-byte load
// of B feeds eight multiply-adds, as it does for N >= 2.
#include "kernels.cuh"

namespace xebk {

namespace {

constexpr int kKeyedThreads = 256;

__device__ __forceinline__ float2 kcfma(float2 acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
    return acc;
}

__device__ __forceinline__ int64_t kscatter(int64_t x, const int8_t* pos, int n) {
    int64_t o = 0;
    for (int i = 0; i < n; ++i)
        if ((x >> i) & 1) o |= int64_t(1) << pos[i];
    return o;
}

// bR[(ub K + k) N + n] = B_ub[k][n] for the kvB distinct right operands
__global__ void k_keyed_pack_b(const __grid_constant__ GemmDesc g, int64_t kvB, const float2* __restrict__ arena,
                               float2* __restrict__ bR) {
    const int64_t KN = g.K * g.N, total = kvB * KN;
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
        const int64_t ub = e / KN, kn = e - ub * KN, k = kn / g.N, n = kn - k * g.N;
        bR[e] = arena[g.b_off + ub * g.b_key + kscatter(k, g.bpk, g.nbk) + kscatter(n, g.bpn, g.nbn)];
    }
}

}  // namespace

template <int K, int N, int RPT>
__global__ void __launch_bounds__(kKeyedThreads) k_gemm_keyed(const __grid_constant__ GemmDesc g,
                                                              float2* __restrict__ arena,
                                                              const float2* __restrict__ bR) {
    constexpr bool kPrefetch = RPT == 1 && K <= 16;   // next item's row in registers
    constexpr int KB = N == 1 ? 2 : 1;                // keys per pass
    constexpr int kRowBits = RPT == 1 ? 5 : 6;        // rows per item: 32 RPT
    __shared__ int64_t rowinc[kMaxLegs];              // address increment of row bit i
    __shared__ int32_t koff[K];                       // address offset of summed index k
    const int tid = threadIdx.x, lane = tid & 31;
    for (int i = tid; i < g.nam; i += kKeyedThreads) rowinc[i] = int64_t(1) << g.apm[i];
    for (int k = tid; k < K; k += kKeyedThreads) koff[k] = int32_t(kscatter(k, g.apk, g.nak));
    __syncthreads();
    int64_t lo = 0;                                   // offset of row bits 0-4 (the lane)
    for (int i = 0; i < 5; ++i)
        if ((lane >> i) & 1) lo += rowinc[i];
    const int64_t rbpg = g.M >> kRowBits;             // row blocks per group
    const int64_t items = g.n_groups * rbpg;
    const int64_t nw = int64_t(gridDim.x) * (kKeyedThreads / 32);
    int64_t item = (int64_t(blockIdx.x) * kKeyedThreads + tid) >> 5;
    // rows rb * 32 RPT + 32 j + lane of the item's group into a[j][.]
    auto load_a = [&](int64_t it, float2 (*dst)[K]) {
        const int64_t grp = it / rbpg, rb = it - grp * rbpg;
        const int64_t u0 = g.gstart ? g.gstart[grp] : 0;
        const int64_t aoff = g.uL ? int64_t(g.uL[u0]) * g.a_key : 0;
        int64_t hi = 0;
        int i = kRowBits;
        for (int64_t x = rb; x != 0; x >>= 1, ++i)
            if (x & 1) hi += rowinc[i];
        const float2* p = arena + g.a_off + aoff + lo + hi;
#pragma unroll
        for (int j = 0; j < RPT; ++j) {
            const float2* pj = p + (j ? rowinc[5] : 0);
#pragma unroll
            for (int k = 0; k < K; ++k) dst[j][k] = __ldg(pj + koff[k]);
        }
    };
    float2 a[RPT][K];
    if (item < items) load_a(item, a);
    for (; item < items; item += nw) {
        float2 an[kPrefetch ? RPT : 1][K];
        const int64_t nxt = item + nw;
        if constexpr (kPrefetch) {
            if (nxt < items) load_a(nxt, an);
        }
        const int64_t grp = item / rbpg, rb = item - grp * rbpg;
        const int64_t u0 = g.gstart ? g.gstart[grp] : 0;
        const int64_t u1 = g.gstart ? g.gstart[grp + 1] : g.kv;
        float2* crow = arena + g.c_off + ((rb << kRowBits) + lane) * N;   // row of j = 0; j adds 32 N
        for (int64_t u = u0; u < u1; u += KB) {
            const float2* b0 = bR + (g.uR ? int64_t(g.uR[u]) : 0) * (K * N);
            if constexpr (KB == 2) {
                const bool two = u + 1 < u1;
                const float2* b1 = two ? bR + (g.uR ? int64_t(g.uR[u + 1]) : 0) * K : b0;
                float2 c0[RPT], c1[RPT];
#pragma unroll
                for (int j = 0; j < RPT; ++j) c0[j] = c1[j] = make_float2(0.f, 0.f);
#pragma unroll
                for (int k = 0; k < K; k += 2) {
                    const float4 q0 = __ldg(reinterpret_cast<const float4*>(b0 + k));
                    const float4 q1 = __ldg(reinterpret_cast<const float4*>(b1 + k));
#pragma unroll
                    for (int j = 0; j < RPT; ++j) {
                        c0[j] = kcfma(c0[j], a[j][k], make_float2(q0.x, q0.y));
                        c0[j] = kcfma(c0[j], a[j][k + 1], make_float2(q0.z, q0.w));
                        c1[j] = kcfma(c1[j], a[j][k], make_float2(q1.x, q1.y));
                        c1[j] = kcfma(c1[j], a[j][k + 1], make_float2(q1.z, q1.w));
                    }
                }
#pragma unroll
                for (int j = 0; j < RPT; ++j) {
                    crow[u * g.c_key + 32 * j] = c0[j];
                    if (two) crow[(u + 1) * g.c_key + 32 * j] = c1[j];
                }
            } else {
                float2 acc[RPT][N];
#pragma unroll
                for (int j = 0; j < RPT; ++j)
#pragma unroll
                    for (int n = 0; n < N; ++n) acc[j][n] = make_float2(0.f, 0.f);
#pragma unroll
                for (int k = 0; k < K; ++k) {
#pragma unroll
                    for (int n = 0; n < N; n += 2) {
                        const float4 q = __ldg(reinterpret_cast<const float4*>(b0 + k * N + n));
#pragma unroll
                        for (int j = 0; j < RPT; ++j) {
                            acc[j][n] = kcfma(acc[j][n], a[j][k], make_float2(q.x, q.y));
                            acc[j][n + 1] = kcfma(acc[j][n + 1], a[j][k], make_float2(q.z, q.w));
                        }
                    }
                }
#pragma unroll
                for (int j = 0; j < RPT; ++j) {
                    float2* c = crow + u * g.c_key + 32 * j * N;
#pragma unroll
                    for (int n = 0; n < N; n += 2)
                        *reinterpret_cast<float4*>(c + n) =
                            make_float4(acc[j][n].x, acc[j][n].y, acc[j][n + 1].x, acc[j][n + 1].y);
                }
            }
        }
        if constexpr (kPrefetch) {
#pragma unroll
            for (int k = 0; k < K; ++k) a[0][k] = an[0][k];
        } else {
            if (nxt < items) load_a(nxt, a);
        }
    }
}

bool keyed_fits(int64_t M, int64_t N, int64_t K) {
    return M >= 32 && M % 32 == 0 && (K == 4 || K == 8 || K == 16 || K == 32) &&
           (N == 1 || N == 2 || N == 4 || N == 8 || N == 16);
}

bool keyed_fits_rows2(int64_t M, int64_t N, int64_t K) { return keyed_fits(M, N, K) && M % 64 == 0 && K <= 16; }

size_t keyed_scratch_bytes(int64_t kvB, int64_t K, int64_t N) { return size_t(kvB * K * N) * sizeof(float2) + 256; }

namespace {
template <int K, int RPT>
void launch_k(const GemmDesc& g, float2* arena, const float2* bR, int grid, cudaStream_t st) {
    switch (g.N) {
        case 1: k_gemm_keyed<K, 1, RPT><<<grid, kKeyedThreads, 0, st>>>(g, arena, bR); break;
        case 2: k_gemm_keyed<K, 2, RPT><<<grid, kKeyedThreads, 0, st>>>(g, arena, bR); break;
        case 4: k_gemm_keyed<K, 4, RPT><<<grid, kKeyedThreads, 0, st>>>(g, arena, bR); break;
        case 8: k_gemm_keyed<K, 8, RPT><<<grid, kKeyedThreads, 0, st>>>(g, arena, bR); break;
        default: k_gemm_keyed<K, 16, RPT><<<grid, kKeyedThreads, 0, st>>>(g, arena, bR); break;
    }
}
}  // namespace

cudaError_t launch_gemm_keyed(const GemmDesc& g, int64_t kvB, int rpt, float2* arena, char* scratch, int n_sms,
                              cudaStream_t st) {
    if (!keyed_fits(g.M, g.N, g.K) || !(rpt == 1 || (rpt == 2 && keyed_fits_rows2(g.M, g.N, g.K))))
        return cudaErrorInvalidValue;
    float2* bR = reinterpret_cast<float2*>(scratch);
    const int64_t nb = kvB * g.K * g.N;
    const int pgrid = int(nb / 256 + 1 < int64_t(n_sms) * 8 ? nb / 256 + 1 : int64_t(n_sms) * 8);
    k_keyed_pack_b<<<pgrid, 256, 0, st>>>(g, kvB, arena, bR);
    const int64_t warps = g.n_groups * (g.M >> (rpt == 1 ? 5 : 6));
    const int64_t want = (warps + 7) / 8;
    const int grid = int(want < int64_t(n_sms) * 8 ? want : int64_t(n_sms) * 8);
    if (rpt == 1) {
        switch (g.K) {
            case 4: launch_k<4, 1>(g, arena, bR, grid, st); break;
            case 8: launch_k<8, 1>(g, arena, bR, grid, st); break;
            case 16: launch_k<16, 1>(g, arena, bR, grid, st); break;
            default: launch_k<32, 1>(g, arena, bR, grid, st); break;
        }
    } else {
        switch (g.K) {
            case 4: launch_k<4, 2>(g, arena, bR, grid, st); break;
            case 8: launch_k<8, 2>(g, arena, bR, grid, st); break;
            default: launch_k<16, 2>(g, arena, bR, grid, st); break;
        }
    }
    return cudaGetLastError();
}

}  // namespace xebk
