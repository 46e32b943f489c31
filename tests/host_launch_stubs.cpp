// Test infrastructure: host-only stand-ins for the CUDA runtime and for the
// library's kernel launchers.  Linked with the library's host sources (the
// planner and the C ABI), a plan binds to a fake device address range, a step
// runs without a GPU, and every launch is written to a text log (the file
// named by XEB_EMU_LOG) with its descriptor: operand offsets, key-table
// pointers, bit positions, launch form.  Device-to-host copies read zeros.
// tests/test_launch_descriptors_host.py checks the logged launches of large
// plans for operand ranges and for the alignment that the kernels' 16-byte
// accesses need.
#include <cuda.h>
#include <cuda_runtime_api.h>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <cstdint>
#include <cinttypes>
#include "kernels.cuh"
#include "xeb.h"

static FILE* logf() {
    static FILE* f = nullptr;
    if (!f) {
        const char* p = getenv("XEB_EMU_LOG");
        f = fopen(p ? p : "/tmp/xeb_emu.log", "w");
    }
    return f;
}
static uintptr_t g_base = uintptr_t(0x100000000000ull);
static uintptr_t g_next = g_base;

extern "C" {
cudaError_t cudaDeviceGetAttribute(int* v, cudaDeviceAttr a, int) {
    if (a == cudaDevAttrMultiProcessorCount) *v = 152;
    else if (a == cudaDevAttrComputeCapabilityMajor) *v = 10;
    else if (a == cudaDevAttrComputeCapabilityMinor) *v = 3;
    else *v = 0;
    return cudaSuccess;
}
cudaError_t cudaGetDevice(int* d) { *d = 0; return cudaSuccess; }
cudaError_t cudaMalloc(void** p, size_t n) {
    *p = reinterpret_cast<void*>(g_next);
    fprintf(logf(), "malloc base=%" PRIuPTR " bytes=%zu\n", g_next - g_base, n);
    g_next += (n + 0xFFFFF) & ~size_t(0xFFFFF);
    return cudaSuccess;
}
cudaError_t cudaFree(void*) { return cudaSuccess; }
cudaError_t cudaMemcpyAsync(void* dst, const void* src, size_t n, cudaMemcpyKind k, cudaStream_t) {
    // device-to-host reads (error words, results) come back as zeros
    if (k == cudaMemcpyDeviceToHost) memset(dst, 0, n);
    (void)src;
    return cudaSuccess;
}
cudaError_t cudaMemsetAsync(void*, int, size_t, cudaStream_t) { return cudaSuccess; }
cudaError_t cudaStreamSynchronize(cudaStream_t) { return cudaSuccess; }
const char* cudaGetErrorString(cudaError_t) { return "emulated"; }
cudaError_t cudaEventCreate(cudaEvent_t* e) { *e = reinterpret_cast<cudaEvent_t>(uintptr_t(1)); return cudaSuccess; }
cudaError_t cudaEventDestroy(cudaEvent_t) { return cudaSuccess; }
cudaError_t cudaEventElapsedTime(float* ms, cudaEvent_t, cudaEvent_t) { *ms = 0.f; return cudaSuccess; }
cudaError_t cudaEventRecord(cudaEvent_t, cudaStream_t) { return cudaSuccess; }
cudaError_t cudaEventRecordWithFlags(cudaEvent_t, cudaStream_t, unsigned int) { return cudaSuccess; }
cudaError_t cudaEventSynchronize(cudaEvent_t) { return cudaSuccess; }
cudaError_t cudaGraphDestroy(cudaGraph_t) { return cudaSuccess; }
cudaError_t cudaGraphExecDestroy(cudaGraphExec_t) { return cudaSuccess; }
cudaError_t cudaGraphInstantiate(cudaGraphExec_t* g, cudaGraph_t, unsigned long long) {
    *g = reinterpret_cast<cudaGraphExec_t>(uintptr_t(1));
    return cudaSuccess;
}
cudaError_t cudaGraphLaunch(cudaGraphExec_t, cudaStream_t) { return cudaSuccess; }
cudaError_t cudaStreamBeginCapture(cudaStream_t, cudaStreamCaptureMode) { return cudaSuccess; }
cudaError_t cudaStreamEndCapture(cudaStream_t, cudaGraph_t* g) {
    *g = reinterpret_cast<cudaGraph_t>(uintptr_t(1));
    return cudaSuccess;
}
cudaError_t cudaStreamCreateWithFlags(cudaStream_t* s, unsigned int) {
    *s = reinterpret_cast<cudaStream_t>(uintptr_t(2));
    return cudaSuccess;
}
cudaError_t cudaStreamDestroy(cudaStream_t) { return cudaSuccess; }
static CUresult fake_encode(CUtensorMap* m, CUtensorMapDataType, cuuint32_t rank, void* addr, const cuuint64_t* dims,
                            const cuuint64_t* strides, const cuuint32_t* box, const cuuint32_t*, CUtensorMapInterleave,
                            CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill) {
    fprintf(logf(), "tmap rank=%u addr=%" PRIuPTR, rank, uintptr_t(addr) - g_base);
    for (cuuint32_t i = 0; i < rank; ++i) fprintf(logf(), " dim%u=%llu", i, (unsigned long long)dims[i]);
    for (cuuint32_t i = 0; i + 1 < rank; ++i) fprintf(logf(), " stride%u=%llu", i, (unsigned long long)strides[i]);
    for (cuuint32_t i = 0; i < rank; ++i) fprintf(logf(), " box%u=%u", i, box[i]);
    fprintf(logf(), "\n");
    memset(m, 0, sizeof(*m));
    return CUDA_SUCCESS;
}
cudaError_t cudaGetDriverEntryPointByVersion(const char*, void** fn, unsigned int, unsigned long long,
                                             cudaDriverEntryPointQueryResult* q) {
    *fn = reinterpret_cast<void*>(&fake_encode);
    if (q) *q = cudaDriverEntryPointSuccess;
    return cudaSuccess;
}
xeb_status xeb_mlp_forward(xeb_mlp_s*, const float*, int, float*, uintptr_t) { return XEB_EUNSUPPORTED; }
xeb_status xeb_mlp_create(int, int, int, uint64_t, xeb_mlp_s**) { return XEB_EUNSUPPORTED; }
void xeb_mlp_destroy(xeb_mlp_s*) {}
size_t xeb_mlp_n_params(xeb_mlp_s*) { return 0; }
xeb_status xeb_mlp_weights(xeb_mlp_s*, float*, int) { return XEB_EUNSUPPORTED; }
xeb_status xeb_mlp_set_norm(xeb_mlp_s*, const float*, const float*) { return XEB_EUNSUPPORTED; }
xeb_status xeb_mlp_gradients(xeb_mlp_s*, const float*, const float*, int, float*, float*, uintptr_t) { return XEB_EUNSUPPORTED; }
xeb_status xeb_mlp_train_step(xeb_mlp_s*, const float*, const float*, int, float, float*, uintptr_t) { return XEB_EUNSUPPORTED; }
xeb_status xeb_linear_xeb_noalloc(const double*, size_t, int, double*, uintptr_t) { return XEB_EUNSUPPORTED; }
}  // extern "C"

namespace xebk {
static long long off(const void* p) { return p ? (long long)(uintptr_t(p) - g_base) : -1; }
static void log_g(const char* kind, const GemmDesc& g, const void* arena) {
    FILE* f = logf();
    fprintf(f, "%s arena=%lld M=%lld N=%lld K=%lld kv=%lld a_off=%lld a_key=%lld b_off=%lld b_key=%lld c_off=%lld c_key=%lld",
            kind, off(arena), (long long)g.M, (long long)g.N, (long long)g.K, (long long)g.kv, (long long)g.a_off,
            (long long)g.a_key, (long long)g.b_off, (long long)g.b_key, (long long)g.c_off, (long long)g.c_key);
    fprintf(f, " nam=%d nak=%d nbk=%d nbn=%d c_natural=%d n_groups=%lld uL=%lld uR=%lld gstart=%lld", g.nam, g.nak, g.nbk,
            g.nbn, g.c_natural, (long long)g.n_groups, off(g.uL), off(g.uR), off(g.gstart));
    fprintf(f, " apm=");
    for (int i = 0; i < g.nam; ++i) fprintf(f, "%d,", g.apm[i]);
    fprintf(f, " apk=");
    for (int i = 0; i < g.nak; ++i) fprintf(f, "%d,", g.apk[i]);
    fprintf(f, " bpk=");
    for (int i = 0; i < g.nbk; ++i) fprintf(f, "%d,", g.bpk[i]);
    fprintf(f, " bpn=");
    for (int i = 0; i < g.nbn; ++i) fprintf(f, "%d,", g.bpn[i]);
    fprintf(f, " cpm=");
    for (int i = 0; i < g.nam; ++i) fprintf(f, "%d,", g.cpm[i]);
    fprintf(f, " cpn=");
    for (int i = 0; i < g.nbn; ++i) fprintf(f, "%d,", g.cpn[i]);
}
cudaError_t prepare_kernels() { return cudaSuccess; }
cudaError_t launch_trie_keys(const TrieDesc*, int n, const uint64_t*, int k, const int32_t*, char* tables, int32_t*,
                             cudaStream_t) {
    fprintf(logf(), "trie_keys n=%d k=%d tables=%lld\n", n, k, off(tables));
    return cudaSuccess;
}
size_t trie_sort_scratch_bytes(int k) {
    const size_t nb = size_t((k + 4096 - 1) / 4096);
    return 2 * size_t(k) * 8 + 2 * size_t(k) * 4 + 256 * nb * 4 + nb * 4 + 4 * 256;
}
cudaError_t launch_trie_keys_large(const TrieDesc*, const TrieDesc* h, int n, const uint64_t*, int k, const int32_t*,
                                   char* tables, char* scratch, int32_t*, cudaStream_t) {
    fprintf(logf(), "trie_keys_large n=%d k=%d tables=%lld scratch=%lld\n", n, k, off(tables), off(scratch));
    for (int i = 0; i < n; ++i)
        fprintf(logf(), "trie_node %d a=%d b=%d kv=%d key_off=%lld uniq_off=%lld rep_off=%lld uL_off=%lld uR_off=%lld gstart_off=%lld kL=%d\n", i,
                h[i].a, h[i].b, h[i].kv, (long long)h[i].key_off, (long long)h[i].uniq_off, (long long)h[i].rep_off,
                (long long)h[i].uL_off, (long long)h[i].uR_off, (long long)h[i].gstart_off, h[i].kL);
    return cudaSuccess;
}
cudaError_t launch_trie_links(const TrieDesc*, const int*, int n, int max_kv, char*, cudaStream_t) {
    fprintf(logf(), "trie_links n=%d max_kv=%d\n", n, max_kv);
    return cudaSuccess;
}
template <typename T>
cudaError_t launch_leaves(const LeafDesc*, int n, const T*, T*, const char*, int64_t slice, cudaStream_t) {
    fprintf(logf(), "leaves n=%d slice=%lld\n", n, (long long)slice);
    return cudaSuccess;
}
template <typename T>
cudaError_t launch_permute(const PermDesc& p, const T* src, T* dst, cudaStream_t) {
    fprintf(logf(), "permute r=%d src=%lld dst=%lld\n", p.r, off(src), off(dst));
    return cudaSuccess;
}
template <typename T>
cudaError_t launch_gemm(int kernel, const GemmDesc& g, T* arena, cudaStream_t) {
    char k[32];
    snprintf(k, sizeof(k), "gemm%d", kernel);
    log_g(k, g, arena);
    fprintf(logf(), " elem=%zu\n", sizeof(T));
    return cudaSuccess;
}
template <typename T>
cudaError_t launch_gemm_stream(const GemmDesc& g, const StreamDesc& s, T* arena, cudaStream_t) {
    log_g("stream", g, arena);
    fprintf(logf(), " elem=%zu R=%d npt=%d T=%d\n", sizeof(T), s.R, s.npt, s.T);
    return cudaSuccess;
}
size_t memo_scratch_bytes(int64_t n_groups, int64_t kv, int64_t K, size_t elem) {
    return size_t(n_groups) * 8 + 256 + size_t(kv * K) * elem;
}
template <typename T>
cudaError_t launch_gemm_memo(const GemmDesc& g, const StreamDesc& s, T* arena, char* scratch, cudaStream_t) {
    log_g("memo", g, arena);
    fprintf(logf(), " elem=%zu R=%d scratch=%lld\n", sizeof(T), s.R, off(scratch));
    return cudaSuccess;
}
template <typename T>
cudaError_t launch_memo_prep(const GemmDesc& g, T* arena, char* scratch, cudaStream_t) {
    log_g("memo_prep", g, arena);
    fprintf(logf(), " scratch=%lld\n", off(scratch));
    return cudaSuccess;
}
template <typename T>
cudaError_t launch_root_accum(const T* root, double2* acc, int64_t kv, cudaStream_t) {
    fprintf(logf(), "root_accum root=%lld acc=%lld kv=%lld\n", off(root), off(acc), (long long)kv);
    return cudaSuccess;
}
cudaError_t launch_gather_xeb(const double2* acc, const int32_t* key_root, int64_t k, const RootMap&, double2* amps,
                              double* partials, int nb, double* result, int, cudaStream_t) {
    fprintf(logf(), "gather_xeb acc=%lld key_root=%lld k=%lld amps=%lld partials=%lld nb=%d result=%lld\n", off(acc),
            off(key_root), (long long)k, off(amps), off(partials), nb, off(result));
    return cudaSuccess;
}
bool keyed_fits(int64_t M, int64_t N, int64_t K) {
    return M >= 32 && M % 32 == 0 && (K == 4 || K == 8 || K == 16 || K == 32) &&
           (N == 1 || N == 2 || N == 4 || N == 8 || N == 16);
}
bool keyed_fits_rows2(int64_t M, int64_t N, int64_t K) { return keyed_fits(M, N, K) && M % 64 == 0 && K <= 16; }
size_t keyed_scratch_bytes(int64_t kvB, int64_t K, int64_t N) { return size_t(kvB * K * N) * sizeof(float2) + 256; }
cudaError_t launch_gemm_keyed(const GemmDesc& g, int64_t kvB, int rpt, float2* arena, char* scratch, int, cudaStream_t) {
    log_g("keyed", g, arena);
    fprintf(logf(), " kvB=%lld rpt=%d scratch=%lld\n", (long long)kvB, rpt, off(scratch));
    return cudaSuccess;
}
cudaError_t launch_tc_gemm2(const TcDesc& t, const CUtensorMap&, float2* arena, int, cudaStream_t) {
    fprintf(logf(), "tc2 arena=%lld M=%lld K2=%d N2=%d tma=%d a_off=%lld b_off=%lld c_off=%lld grp=%d\n", off(arena),
            (long long)t.M, t.K2, t.N2, t.tma, (long long)t.a_off, (long long)t.b_off, (long long)t.c_off, t.grp);
    return cudaSuccess;
}
cudaError_t launch_tc_kdeep(const KdDesc& d, float2* arena, int, cudaStream_t) {
    fprintf(logf(), "tckd arena=%lld M=%d N=%d K=%d kv=%lld a_off=%lld a_key=%lld b_off=%lld b_key=%lld c_off=%lld c_key=%lld n_groups=%lld\n",
            off(arena), d.M, d.N, d.K, (long long)d.kv, (long long)d.a_off, (long long)d.a_key, (long long)d.b_off,
            (long long)d.b_key, (long long)d.c_off, (long long)d.c_key, (long long)d.n_groups);
    return cudaSuccess;
}
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
template cudaError_t launch_memo_prep<float2>(const GemmDesc&, float2*, char*, cudaStream_t);
template cudaError_t launch_root_accum<float2>(const float2*, double2*, int64_t, cudaStream_t);
template cudaError_t launch_root_accum<double2>(const double2*, double2*, int64_t, cudaStream_t);
}  // namespace xebk
