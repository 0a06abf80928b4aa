// noalloc.cu -- vloc_apply_noalloc: the V_loc apply with no allocation.
//
// Some callers cannot call cudaMalloc: code that runs while another runtime
// owns the device's memory (a framework that reserves the GPU's memory up
// front and forbids outside allocations), or a process that must never
// allocate after start-up.  For them this file holds the scratch the apply
// needs -- index tables, twiddles, the cylinder and the slab -- in one
// fixed, file-scope device array instead of the plan's workspace.  It works
// with any complex (non-Gamma) plan, including a VLOC_HOST_ONLY plan (which
// itself made no CUDA call), so the pair vloc_plan_create(VLOC_HOST_ONLY) +
// vloc_apply_noalloc never allocates device memory.
//
// The array is kScratchBytes (48 MiB) per GPU that loads this library, held
// until the process exits.  Every call shares it and leaves its contents
// behind; nothing in it has to start at zero (every element is written
// before it is read), so no clearing is needed.  Calls that overlap on the
// GPU (two streams, or two host threads whose work interleaves) race on the
// array: serialise them.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/vloc.h"
#include "internal.h"

namespace {

constexpr size_t kScratchBytes = (size_t)48 << 20;   // device scratch per GPU
constexpr size_t kTableInts = (size_t)2 << 20;       // index tables at most 8 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_vloc_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};  // device address of g_vloc_scratch, per device

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }
bool overlap(const void* a, size_t na, const void* b, size_t nb) {
    const char *pa = (const char*)a, *pb = (const char*)b;
    return pa < pb + nb && pb < pa + na;
}

}  // namespace

extern "C" int vloc_apply_noalloc(vloc_plan plan, const void* coeffs, const void* V, int64_t nbands, void* out,
                                  void* stream) {
    using namespace vloc;
    if (!plan || nbands < 0) return VLOC_ERR_ARG;
    vloc_info info;
    int rc = vloc_get_info(plan, &info);
    if (rc) return rc;
    // Gamma-point plans keep half-list coefficients and need the pack /
    // unpack buffers of the plan's workspace: not offered here.  Checked
    // before anything else, so no CUDA call is made for them.
    if (info.path & 4) return VLOC_ERR_STATE;
    if (nbands == 0) return VLOC_OK;
    if (!coeffs || !V || !out) return VLOC_ERR_ARG;
    const int dbl = info.precision == VLOC_F64;
    const int fast = (info.path & 8) ? 2 : (info.path & 1);  // the plan's own kernel family
    const size_t elem = dbl ? 16 : 8, re = dbl ? 8 : 4;
    if ((uintptr_t)coeffs % elem || (uintptr_t)out % elem || (uintptr_t)V % re) return VLOC_ERR_ARG;
    const size_t bytes = (size_t)nbands * (size_t)info.npw * elem;
    const long long N = (long long)info.n1 * info.n2 * info.n3;
    if (coeffs != out && overlap(coeffs, bytes, out, bytes)) return VLOC_ERR_ARG;
    if (overlap(V, (size_t)N * re, out, bytes)) return VLOC_ERR_ARG;

    const int* host_tables = nullptr;
    HostTableLayout lay;
    rc = plan_host_tables(plan, &host_tables, &lay);
    if (rc) return rc;
    if (lay.total > kTableInts) return VLOC_ERR_SIZE;

    // scratch layout: tables | twiddles per axis | (double-float: TwDF per
    // axis, V as hi + lo pairs) | cylinder chunk | slab chunk
    const size_t tab_bytes = up256(lay.total * sizeof(int));
    const int ns[3] = {info.n1, info.n2, info.n3};
    size_t tw_off[3], twdf_off[3] = {0, 0, 0}, vdf_off = 0, off = tab_bytes;
    for (int a = 0; a < 3; ++a) { tw_off[a] = off; off += up256((size_t)ns[a] * elem); }
    if (fast == 2) {
        for (int a = 0; a < 3; ++a) { twdf_off[a] = off; off += up256((size_t)ns[a] * 32); }
        vdf_off = off;
        off += up256((size_t)N * 8);
    }
    const size_t cyl_band = (size_t)lay.S * info.n3 * elem;
    const size_t slab_band = (size_t)lay.NP * info.n2 * info.n3 * elem;
    if (off + up256(cyl_band) + up256(slab_band) > kScratchBytes) return VLOC_ERR_SIZE;
    long long chunk = 1;
    while (chunk < 65535 && off + up256((size_t)(chunk + 1) * cyl_band) + up256((size_t)(chunk + 1) * slab_band) <= kScratchBytes)
        ++chunk;

    std::lock_guard<std::mutex> lock(g_mu);
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return VLOC_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return VLOC_ERR_ARG;
    // Set-up, once per device, with that device current: the host-side name
    // g_vloc_scratch is only a stand-in, the kernels need the device address.
    if (!g_scratch_addr[dev]) {
        void* addr = nullptr;
        e = cudaGetSymbolAddress(&addr, g_vloc_scratch);
        if (e != cudaSuccess || !addr) return VLOC_ERR_CUDA;
        g_scratch_addr[dev] = addr;
    }
    char* base = (char*)g_scratch_addr[dev];
    char* cyl = base + off;
    char* slab = cyl + up256((size_t)chunk * cyl_band);

    int optin = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return VLOC_ERR_CUDA;
    int nmax = info.n1 > info.n2 ? info.n1 : info.n2;
    if (info.n3 > nmax) nmax = info.n3;
    if (smem_bytes_for(dbl, nmax) > (size_t)optin) return VLOC_ERR_SIZE;
    if (set_smem_limits(dbl, nmax, optin)) return VLOC_ERR_CUDA;

    // the plan's own host table block (unchanged for the plan's life) -> scratch
    if (cudaMemcpyAsync(base, host_tables, lay.total * sizeof(int), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return VLOC_ERR_CUDA;
    for (int a = 0; a < 3; ++a)
        if (launch_twiddles(dbl, base + tw_off[a], ns[a], st)) return VLOC_ERR_CUDA;
    const void* tw[3] = {base + tw_off[0], base + tw_off[1], base + tw_off[2]};
    const void* Vk = V;
    if (fast == 2) {
        for (int a = 0; a < 3; ++a) {
            if (launch_twiddles_df(base + tw_off[a], base + twdf_off[a], ns[a], st)) return VLOC_ERR_CUDA;
            tw[a] = base + twdf_off[a];
        }
        if (launch_v_to_df(V, base + vdf_off, N, st)) return VLOC_ERR_CUDA;
        Vk = base + vdf_off;
    }

    const DevTables t = device_tables((const int*)base, lay, info.n1, info.n2, info.n3, info.npw);
    LaunchAxes ax;
    for (int a = 0; a < 3; ++a) {
        ax.n[a] = ns[a];
        ax.nst[a] = info.nstages[a];
        for (int i = 0; i < 4; ++i) ax.radix[a][i] = info.radix[a][i];
    }
    const size_t bstride = (size_t)info.npw * elem;
    for (int64_t b0 = 0; b0 < nbands; b0 += chunk) {
        const long long cb = nbands - b0 < chunk ? nbands - b0 : chunk;
        const void* cc = (const char*)coeffs + b0 * bstride;
        void* oo = (char*)out + b0 * bstride;
        if (launch_k1_scatter_zpass(dbl, fast, t, ax, tw[2], cc, cb, cyl, st)) return VLOC_ERR_CUDA;
        if (launch_k2_ypass(dbl, fast, +1, t, ax, tw[1], cb, cyl, slab, st)) return VLOC_ERR_CUDA;
        if (launch_k3_xpass_v(dbl, fast, t, ax, tw[0], Vk, cb, slab, st)) return VLOC_ERR_CUDA;
        if (launch_k2_ypass(dbl, fast, -1, t, ax, tw[1], cb, cyl, slab, st)) return VLOC_ERR_CUDA;
        if (launch_k4_zpass_gather(dbl, fast, t, ax, tw[2], cyl, cb, oo, nullptr, nullptr, st)) return VLOC_ERR_CUDA;
    }
    return VLOC_OK;
}
