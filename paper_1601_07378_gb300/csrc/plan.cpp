// plan.cpp -- host plan builder and the C ABI of include/vloc.h.
//
// A plan turns a grid and a plane-wave list into the index tables the
// kernels walk (Sec. 2 Eqs. 2-3: each G is one grid point; Sec. 4.3 /
// Fig. 5: the occupied sticks form the cylinder, the occupied x-planes the
// cuboid), deals the sticks to z-pass thread blocks with the paper's greedy
// sorted round-robin (Sec. 3.2, Fig. 2) or one of its row/column schemes
// (Sec. 4.1, 4.2), makes the twiddles on the device in FP64 and owns the
// workspace that replaces the distributed FFT's transposes.
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <numeric>
#include <vector>

#include "../../include/vloc.h"
#include "internal.h"

using namespace vloc;

namespace {

thread_local char g_last_cuda[256] = "";

int cuda_fail(cudaError_t e, const char* what) {
    snprintf(g_last_cuda, sizeof(g_last_cuda), "%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? VLOC_ERR_ALLOC : VLOC_ERR_CUDA;
}
#define CK(call)                                              \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);   \
    } while (0)

const int kRadices[] = {16, 15, 12, 10, 9, 8, 6, 5, 4, 3, 2};
constexpr long long kGradBandsPerGroup = 16;

// Host-buffer apply: bands per staging chunk, and the growth (x2) of the
// ramps of smaller chunks at both ends (4: doubling; 2 or less: no ramp).
#ifndef VLOC_STAGE_BANDS
#define VLOC_STAGE_BANDS 256
#endif
#ifndef VLOC_STAGE_RAMP
#define VLOC_STAGE_RAMP 4
#endif
// staging slots (chunks in flight between copy in, compute and copy out), <= 4
#ifndef VLOC_STAGE_SLOTS
#define VLOC_STAGE_SLOTS 2
#endif
constexpr long long kBatchBranches = 4;  // parallel branches of a batched graph  // bands per group of the dL/dV x-pass (FP32 sums)
constexpr int kLinesPerTile = 32;

bool smooth235(int n) {
    for (int p : {2, 3, 5})
        while (n % p == 0) n /= p;
    return n == 1;
}

// Fewest stages, then the smallest largest radix, then larger radices first.
bool plan_radices(int n, int* nst, int radix[4]) {
    for (int r : kRadices)
        if (r == n) { *nst = 1; radix[0] = n; radix[1] = radix[2] = radix[3] = 0; return true; }
    for (int k = 2; k <= 4; ++k) {
        std::vector<int> best;
        int idx[4] = {0, 0, 0, 0};
        const int nr = (int)(sizeof(kRadices) / sizeof(int));
        while (true) {
            long long prod = 1;
            for (int i = 0; i < k; ++i) prod *= kRadices[idx[i]];
            if (prod == n) {
                std::vector<int> c(k);
                for (int i = 0; i < k; ++i) c[i] = kRadices[idx[i]];
                auto key = [](const std::vector<int>& v) {
                    int mx = *std::max_element(v.begin(), v.end());
                    std::vector<int> neg(v.size());
                    for (size_t i = 0; i < v.size(); ++i) neg[i] = -v[i];
                    return std::make_pair(mx, neg);
                };
                if (best.empty() || key(c) < key(best)) best = c;
            }
            int i = k - 1;
            while (i >= 0 && ++idx[i] == nr) { idx[i] = 0; --i; }
            if (i < 0) break;
        }
        if (!best.empty()) {
            *nst = k;
            for (int i = 0; i < 4; ++i) radix[i] = i < k ? best[i] : 0;
            return true;
        }
    }
    return false;
}

int pmod(int a, int n) { int r = a % n; return r < 0 ? r + n : r; }
bool valid_miller(int h, int n) { return h >= -(n / 2) && h <= (n + 1) / 2 - 1; }

// Sec. 4.1: p = m x n with |m - n| minimal, m >= n.
void process_grid(int p, int* m, int* n) {
    int mm = (int)std::ceil(std::sqrt((double)p));
    while (p % mm) ++mm;
    *m = mm;
    *n = p / mm;
}

// Test aids, read from the environment variable VLOC_FAULT when a plan is
// created (unset in normal use):
//   "alloc" or "alloc:K" -- allocation K of vloc_plan_create (0 = the host
//       plan object, 1, 2, ... = its device allocations in order) fails as
//       if memory were exhausted, so every clean-up path can be exercised
//       without exhausting a GPU;
//   "tma_wait" -- the persistent TMA x-pass of the plan never issues the
//       first tile load of its first thread block, so that block's bounded
//       wait runs out and the kernel reports it through the error flag.
struct FaultSpec {
    int alloc_at = -1;
    bool tma_wait = false;
};
FaultSpec fault_spec() {
    FaultSpec f;
    const char* v = std::getenv("VLOC_FAULT");
    if (!v) return f;
    if (std::strncmp(v, "alloc", 5) == 0) f.alloc_at = v[5] == ':' ? std::atoi(v + 6) : 0;
    if (std::strcmp(v, "tma_wait") == 0) f.tma_wait = true;
    return f;
}

}  // namespace

struct vloc_plan_s {
    int n1 = 0, n2 = 0, n3 = 0, dbl = 0, flags = 0;
    long long npw = 0, N = 0;
    int S = 0, NP = 0, P = 0, T = 0;
    int fast = 1;  // compile-time-length kernels where available
    bool df = false;            // FP64 apply in double-float arithmetic
    void* d_twdf[3] = {nullptr, nullptr, nullptr};  // TwDF tables per axis
    void* d_vdf = nullptr;      // V as hi + lo pairs [N]
    int* d_err = nullptr;       // set by a kernel whose bounded wait ran out
    bool k3tma_on = false;      // x-pass through the persistent TMA kernel
    bool poison = false;        // VLOC_POISON_WORKSPACE: NaN-fill before every chunk
    bool gfused = false;        // Gamma pairs formed and separated inside the z-passes
    vloc::K3Tma k3tma{};
    bool gamma = false;       // Gamma-point real mode (half-sphere coefficients)
    long long npw_user = 0;   // plane waves per band in the caller's arrays
    int* d_gamma_neg = nullptr;  // full-list index of -G for each caller G
    void* d_gamma_buf = nullptr; // packed pairs and their results, [2][chunk][npw]
    int ngroups = 1;  // band groups of the dL/dV x-pass
    long long chunk = 1, ws_bands = 2;
    size_t elem = 8;
    LaunchAxes ax{};
    std::vector<int64_t> grid_index;  // caller order
    std::vector<int32_t> stick_part;  // canonical stick order
    std::vector<int> host_tables;     // index tables as uploaded (layout `lay`)
    HostTableLayout lay{};
    // device
    int* d_tables = nullptr;
    DevTables dt{};
    void* d_tw[3] = {nullptr, nullptr, nullptr};
    void* d_cyl = nullptr;
    void* d_slab = nullptr;
    double* d_acc = nullptr;
    size_t ws_bytes = 0;
    // host-buffer path (allocated on first use)
    void* d_stage = nullptr;
    size_t stage_bytes = 0;
    long long stage_bands = 0;
    cudaStream_t copy_stream = nullptr;  // host-to-device copies
    cudaStream_t d2h_stream = nullptr;   // device-to-host copies
    cudaEvent_t ev[12] = {};  // host-buffer staging: 3 events per staging slot
    bool stage_used[4] = {};  // slot s has recorded its computed / copied-out events
    int stage_next = 0;       // slot of the next chunk (kept across calls)
    int device = 0;
    int smem_optin = 0;
    std::mutex mu;
    // CUDA graphs of apply chains (VLOC_GRAPH), keyed by the call's pointers
    struct GraphEntry {
        std::vector<uintptr_t> key;
        cudaGraphExec_t exec = nullptr;
        std::vector<std::pair<vloc_plan_s*, long long>> kernels;  // kernels per plan in the graph
        unsigned long long last_use = 0;
    };
    std::vector<GraphEntry> graphs;
    cudaStream_t cap_stream = nullptr;
    unsigned long long use_clock = 0;
    std::vector<cudaStream_t> branch_streams;  // parallel branches of batched graphs
    std::vector<cudaEvent_t> branch_events;
    cudaEvent_t fork_event = nullptr;
    // launch accounting and optional per-launch event timing
    long long launches = 0;
    bool prof_on = false;
    std::vector<cudaEvent_t> prof_pool;
    std::vector<std::pair<int, size_t>> prof_recs;  // (kind, index of start event)
};

extern "C" {

const char* vloc_strerror(int code) {
    switch (code) {
        case VLOC_OK: return "ok";
        case VLOC_ERR_ARG: return "invalid argument (null or misaligned pointer, bad count or overlap)";
        case VLOC_ERR_SIZE: return "unsupported size (grid must be 2..256 and 2/3/5-smooth)";
        case VLOC_ERR_GLIST: return "invalid G-list (index out of range or duplicate)";
        case VLOC_ERR_ALLOC: return "allocation failed";
        case VLOC_ERR_CUDA: return "CUDA runtime error";
        case VLOC_ERR_TIMEOUT: return "device-side wait timed out";
        case VLOC_ERR_STATE: return "call not allowed by the plan's flags";
        default: return "unknown error";
    }
}

int vloc_version(void) { return 100; }

const char* vloc_last_cuda_error(void) { return g_last_cuda; }

static void free_plan(vloc_plan p) {
    if (!p) return;
    cudaFree(p->d_tables);
    for (void* t : p->d_tw) cudaFree(t);
    cudaFree(p->d_cyl);
    cudaFree(p->d_slab);
    cudaFree(p->d_acc);
    cudaFree(p->d_gamma_neg);
    for (int a = 0; a < 3; ++a) cudaFree(p->d_twdf[a]);
    cudaFree(p->d_vdf);
    cudaFree(p->d_err);
    cudaFree(p->d_gamma_buf);
    cudaFree(p->d_stage);
    for (cudaEvent_t e : p->prof_pool) cudaEventDestroy(e);
    for (auto& g : p->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
    for (cudaStream_t b : p->branch_streams) cudaStreamDestroy(b);
    for (cudaEvent_t b : p->branch_events) cudaEventDestroy(b);
    if (p->fork_event) cudaEventDestroy(p->fork_event);
    for (cudaEvent_t e : p->ev)
        if (e) cudaEventDestroy(e);
    if (p->copy_stream) cudaStreamDestroy(p->copy_stream);
    if (p->d2h_stream) cudaStreamDestroy(p->d2h_stream);
    delete p;
}

int vloc_plan_create(vloc_plan* out, int n1, int n2, int n3, const int32_t* g, int64_t npw, int flags,
                     int64_t max_bands_per_chunk, void* stream) {
    if (!out) return VLOC_ERR_ARG;
    *out = nullptr;
    if (!g || npw <= 0) return npw == 0 ? VLOC_ERR_GLIST : VLOC_ERR_ARG;
    const int prec = flags & (VLOC_F32 | VLOC_F64);
    if (prec != VLOC_F32 && prec != VLOC_F64) return VLOC_ERR_ARG;
    const int part_flag = flags & 0x0F0;
    if (part_flag != VLOC_PARTITION_GREEDY && part_flag != VLOC_PARTITION_BASIC && part_flag != VLOC_PARTITION_IMPROVED)
        return VLOC_ERR_ARG;
    if (flags & ~(0x003 | 0x0F0 | VLOC_GRAPH | VLOC_HOST_ONLY | VLOC_GENERIC_KERNELS | VLOC_GAMMA | VLOC_DOUBLE_FLOAT |
                  VLOC_X_TMA | VLOC_POISON_WORKSPACE | VLOC_Z_WARP | VLOC_Z_BULK))
        return VLOC_ERR_ARG;
    if ((flags & VLOC_DOUBLE_FLOAT) && prec != VLOC_F64) return VLOC_ERR_ARG;
    const bool host_only = (flags & VLOC_HOST_ONLY) != 0;
    const int ns[3] = {n1, n2, n3};
    for (int a = 0; a < 3; ++a)
        if (ns[a] < 2 || ns[a] > 256 || !smooth235(ns[a])) return VLOC_ERR_SIZE;
    // Gamma-point real mode (Sec. 4.3, last paragraph): the caller gives half
    // of a sphere symmetric under G -> -G; the plan runs on the full list
    // (the half, then -G for every G != 0 in the half's order).
    const int64_t npw_user = npw;
    std::vector<int32_t> gfull;
    std::vector<int32_t> gamma_neg;
    if (flags & VLOC_GAMMA) {
        gfull.assign(g, g + 3 * npw);
        gamma_neg.resize(npw);
        int64_t next = npw;
        for (int64_t q = 0; q < npw; ++q) {
            const int h = g[3 * q], k = g[3 * q + 1], l = g[3 * q + 2];
            if (h == 0 && k == 0 && l == 0) { gamma_neg[q] = (int32_t)q; continue; }
            if (!valid_miller(-h, n1) || !valid_miller(-k, n2) || !valid_miller(-l, n3)) return VLOC_ERR_GLIST;
            gfull.insert(gfull.end(), {-h, -k, -l});
            gamma_neg[q] = (int32_t)next++;
        }
        g = gfull.data();
        npw = next;  // duplicates (G and -G both in the half) are caught below
    }
    const long long N = (long long)n1 * n2 * n3;
    if (npw > N) return VLOC_ERR_GLIST;
    const int dbl = prec == VLOC_F64;
    const size_t elem = dbl ? 16 : 8;
    const int nmax = std::max(n1, std::max(n2, n3));

    const FaultSpec fault = fault_spec();
    int alloc_no = 0;  // allocations so far (fault injection counts them)
    vloc_plan p = fault.alloc_at == alloc_no++ ? nullptr : new (std::nothrow) vloc_plan_s();
    if (!p) return VLOC_ERR_ALLOC;
    auto dmalloc = [&](void** ptr, size_t bytes) -> cudaError_t {
        if (fault.alloc_at == alloc_no++) return cudaErrorMemoryAllocation;
        return cudaMalloc(ptr, bytes);
    };
    p->poison = (flags & VLOC_POISON_WORKSPACE) != 0;
    p->n1 = n1; p->n2 = n2; p->n3 = n3; p->dbl = dbl; p->flags = flags; p->npw = npw; p->N = N;
    p->npw_user = npw_user;
    p->gamma = (flags & VLOC_GAMMA) != 0;
    p->elem = elem;
    p->fast = (flags & VLOC_GENERIC_KERNELS) ? 0 : 1;
    p->df = (flags & VLOC_DOUBLE_FLOAT) && !(flags & VLOC_GENERIC_KERNELS) && has_df(n1) && has_df(n2) && has_df(n3);
    for (int a = 0; a < 3; ++a) {
        p->ax.n[a] = ns[a];
        if (!plan_radices(ns[a], &p->ax.nst[a], p->ax.radix[a])) { free_plan(p); return VLOC_ERR_SIZE; }
    }

    // ---- index map and validation (Eqs. 2-3)
    p->grid_index.resize(npw);
    {
        std::vector<unsigned char> seen((size_t)N, 0);
        for (int64_t q = 0; q < npw; ++q) {
            const int h = g[3 * q], k = g[3 * q + 1], l = g[3 * q + 2];
            if (!valid_miller(h, n1) || !valid_miller(k, n2) || !valid_miller(l, n3)) { free_plan(p); return VLOC_ERR_GLIST; }
            const long long j = ((long long)pmod(h, n1) * n2 + pmod(k, n2)) * n3 + pmod(l, n3);
            if (seen[(size_t)j]) { free_plan(p); return VLOC_ERR_GLIST; }
            seen[(size_t)j] = 1;
            p->grid_index[q] = j;
        }
    }
    // ---- canonical order: by stick id (h mod n1) n2 + (k mod n2), then l
    std::vector<int> order(npw);
    std::iota(order.begin(), order.end(), 0);
    auto stick_of = [&](int q) { return (long long)pmod(g[3 * q], n1) * n2 + pmod(g[3 * q + 1], n2); };
    std::sort(order.begin(), order.end(), [&](int a, int b) {
        const long long sa = stick_of(a), sb = stick_of(b);
        if (sa != sb) return sa < sb;
        return g[3 * a + 2] < g[3 * b + 2];
    });
    std::vector<int> pw_user(npw), pw_z(npw), stick_pw_ptr, stick_row, stick_x;
    std::vector<long long> stick_id;
    for (int64_t i = 0; i < npw; ++i) {
        const int q = order[i];
        pw_user[i] = q;
        pw_z[i] = pmod(g[3 * q + 2], n3);
        const long long sid = stick_of(q);
        if (stick_id.empty() || stick_id.back() != sid) {
            stick_id.push_back(sid);
            stick_pw_ptr.push_back((int)i);
            stick_row.push_back((int)(sid % n2));
            stick_x.push_back((int)(sid / n2));
        }
    }
    const int S = (int)stick_id.size();
    stick_pw_ptr.push_back((int)npw);
    // ---- planes (the cuboid of Fig. 5): occupied x = h mod n1
    std::vector<int> plane_ptr, xrow_plane(n1, -1);
    for (int s = 0; s < S; ++s)
        if (s == 0 || stick_x[s] != stick_x[s - 1]) {
            xrow_plane[stick_x[s]] = (int)plane_ptr.size();
            plane_ptr.push_back(s);
        }
    const int NP = (int)plane_ptr.size();
    plane_ptr.push_back(S);

    // ---- partition of the sticks over z-pass thread blocks
    int P = (S + kLinesPerTile - 1) / kLinesPerTile;
    std::vector<int32_t> part(S);
    std::vector<int> weight(S);
    for (int s = 0; s < S; ++s) weight[s] = stick_pw_ptr[s + 1] - stick_pw_ptr[s];
    if (part_flag == VLOC_PARTITION_GREEDY) {
        // Sec. 3.2 / Fig. 2: sort by workload (#PW) descending, ties by stick
        // id ascending; the k-th sorted stick goes to part k mod P.
        std::vector<int> srt(S);
        std::iota(srt.begin(), srt.end(), 0);
        std::stable_sort(srt.begin(), srt.end(), [&](int a, int b) {
            if (weight[a] != weight[b]) return weight[a] > weight[b];
            return stick_id[a] < stick_id[b];
        });
        if (!(flags & VLOC_GAMMA)) {
            for (int r = 0; r < S; ++r) part[srt[r]] = r % P;
        } else {
            // Gamma-point plans deal a stick and its mirror (-h, -k) together
            // (Sec. 4.3: c(-G) = conj c(G) pairs them), so that one z-pass
            // block holds both G and -G of every plane wave it owns.  The same
            // rule on pairs: weight descending, ties by the smaller stick id,
            // the k-th pair to part k mod P, at most 16 pairs per part.
            std::vector<int> mirror(S);
            for (int s2 = 0; s2 < S; ++s2) {
                const long long a = stick_id[s2] / n2, bb = stick_id[s2] % n2;
                const long long mid = ((n1 - a) % n1) * n2 + (n2 - bb) % n2;
                const auto it = std::lower_bound(stick_id.begin(), stick_id.end(), mid);
                mirror[s2] = (it != stick_id.end() && *it == mid) ? (int)(it - stick_id.begin()) : -1;
            }
            std::vector<int> pairs;  // first stick of each pair, in sorted order
            for (int r = 0; r < S; ++r) {
                const int s2 = srt[r], m = mirror[s2];
                if (m < 0 || s2 <= m) pairs.push_back(s2);
                else if (mirror[m] != s2) pairs.push_back(s2);
            }
            P = std::max(P, (int)((pairs.size() + kLinesPerTile / 2 - 1) / (kLinesPerTile / 2)));
            for (size_t r = 0; r < pairs.size(); ++r) {
                const int s2 = pairs[r], m = mirror[s2];
                part[s2] = (int32_t)(r % P);
                if (m >= 0) part[m] = (int32_t)(r % P);
            }
        }
    } else {
        int m, ncol;
        process_grid(P, &m, &ncol);
        std::vector<long long> row_of(n1), col_of(n2);
        if (part_flag == VLOC_PARTITION_BASIC) {
            // Sec. 4.1: cyclic row groups by x, column groups by y.
            for (int a = 0; a < n1; ++a) row_of[a] = a % m;
            for (int b = 0; b < n2; ++b) col_of[b] = b % ncol;
        } else {
            // Sec. 4.2: planes sorted by #PW (descending, ties by index) dealt
            // round-robin to row groups (x-planes) and column groups (y-planes).
            std::vector<long long> wa(n1, 0), wb(n2, 0);
            for (int s = 0; s < S; ++s) { wa[stick_x[s]] += weight[s]; wb[stick_row[s]] += weight[s]; }
            std::vector<int> ia(n1), ib(n2);
            std::iota(ia.begin(), ia.end(), 0);
            std::iota(ib.begin(), ib.end(), 0);
            std::stable_sort(ia.begin(), ia.end(), [&](int a, int b) { return wa[a] != wa[b] ? wa[a] > wa[b] : a < b; });
            std::stable_sort(ib.begin(), ib.end(), [&](int a, int b) { return wb[a] != wb[b] ? wb[a] > wb[b] : a < b; });
            for (int r = 0; r < n1; ++r) row_of[ia[r]] = r % m;
            for (int r = 0; r < n2; ++r) col_of[ib[r]] = r % ncol;
        }
        for (int s = 0; s < S; ++s) part[s] = (int32_t)(row_of[stick_x[s]] * ncol + col_of[stick_row[s]]);
    }
    // ---- tiles: each part's sticks (ascending id) in runs of at most 32
    // lines; one z-pass CTA per tile.  With the greedy partition every part is
    // exactly one tile.  Per tile, the flat list of its plane waves as
    // {caller index, z | line << 16}, sticks in tile order, l ascending.
    std::vector<int> tile_ptr(1, 0), tile_sticks;
    tile_sticks.reserve(S);
    {
        std::vector<std::vector<int>> members(P);
        for (int s = 0; s < S; ++s) members[part[s]].push_back(s);
        for (int q = 0; q < P; ++q)
            for (size_t i = 0; i < members[q].size(); i += kLinesPerTile) {
                const size_t e = std::min(members[q].size(), i + (size_t)kLinesPerTile);
                tile_sticks.insert(tile_sticks.end(), members[q].begin() + i, members[q].begin() + e);
                tile_ptr.push_back((int)tile_sticks.size());
            }
    }
    const int T = (int)tile_ptr.size() - 1;
    std::vector<int> tile_pw_ptr(T + 1, 0), tile_pw;
    tile_pw.reserve(2 * (size_t)npw);
    for (int tt = 0; tt < T; ++tt) {
        for (int i = tile_ptr[tt]; i < tile_ptr[tt + 1]; ++i) {
            const int s = tile_sticks[i], line = i - tile_ptr[tt];
            for (int q = stick_pw_ptr[s]; q < stick_pw_ptr[s + 1]; ++q) {
                tile_pw.push_back(pw_user[q]);
                tile_pw.push_back(pw_z[q] | (line << 16));
            }
        }
        tile_pw_ptr[tt + 1] = (int)(tile_pw.size() / 2);
    }
    p->S = S; p->NP = NP; p->P = P; p->T = T;
    p->stick_part = part;

    // ---- dense z-band table for the z-pass that loads each first-stage input
    // itself (plain plans): per tile, for every row x = i + r NA (NA = n3 /
    // R0, R0 the first radix of the n3 schedule) of a row group r that meets
    // the band |l| <= n3/4, and every line of the tile, the caller index of
    // the plane wave there, or -1.  Rows [tile][group j][i][line], groups in
    // r order.
    std::vector<int> zdense;
    int zd_rows = 0;
    {
        const int R0 = p->ax.radix[2][0], Q3 = n3 / 4;
        const int NA3 = R0 > 0 ? n3 / R0 : 0;
        std::vector<int> groups;
        if (p->ax.nst[2] == 2 && Q3 >= 1 && NA3 > 0)
            for (int r = 0; r < R0; ++r) {
                const int lo = r * NA3, hi = r * NA3 + NA3 - 1;
                if (hi <= Q3 || lo >= n3 - Q3 || lo <= Q3 || hi >= n3 - Q3) groups.push_back(r);
            }
        bool band = !groups.empty() && !(flags & VLOC_GAMMA);
        for (int64_t q = 0; band && q < npw; ++q) band = pw_z[q] <= Q3 || pw_z[q] >= n3 - Q3;
        if (band) {
            std::vector<int> slot_of_row(n3, -1);
            for (size_t j = 0; j < groups.size(); ++j)
                for (int i = 0; i < NA3; ++i) slot_of_row[i + groups[j] * NA3] = (int)(j * NA3 + i);
            zd_rows = (int)groups.size() * NA3;
            zdense.assign((size_t)T * zd_rows * kLinesPerTile, -1);
            for (int tt = 0; tt < T; ++tt)
                for (int e = tile_pw_ptr[tt]; e < tile_pw_ptr[tt + 1]; ++e) {
                    const int f = tile_pw[2 * e], zl = tile_pw[2 * e + 1];
                    const int z = zl & 0xffff, line = zl >> 16;
                    zdense[((size_t)tt * zd_rows + slot_of_row[z]) * kLinesPerTile + line] = f;
                }
        }
    }

    // ---- class table for the warp-register z-passes (VLOC_Z_WARP; plain
    // FP32 plans, n3 = 32 C with C <= 4): per stick, the caller index of the
    // plane wave at z = C m + j in entry 32 j + m, or -1
    std::vector<int> zsh;
    int zs_ok = 0;
    if ((flags & VLOC_Z_WARP) && !(flags & VLOC_GAMMA) && !dbl && n3 % 32 == 0 && n3 / 32 >= 1 && n3 / 32 <= 4) {
        const int C = n3 / 32;
        zsh.assign((size_t)S * n3, -1);
        for (int s = 0; s < S; ++s)
            for (int q = stick_pw_ptr[s]; q < stick_pw_ptr[s + 1]; ++q) {
                const int z = pw_z[q];
                zsh[(size_t)s * n3 + 32 * (z % C) + z / C] = pw_user[q];
            }
        zs_ok = 1;
    }

    // ---- stick runs: plain FP32 quarter-band plans (the dense table exists)
    // whose every stick holds consecutive caller indices in l order with no
    // gap in l (the canonical order); per tile line {first caller index, its
    // l, count, 0}.  K1 then addresses its inputs from the runs (runs = 2;
    // 0.372 against 0.384 ms per 1024 bands at 96^3 through the dense table),
    // or stages them by bulk copies with VLOC_Z_BULK (runs = 1).
    std::vector<int> run_tab;
    int runs_ok = 0;
    if (!(flags & VLOC_Z_WARP) && !dbl && zd_rows > 0) {
        bool ok = true;
        std::vector<int> first(S), lmin(S), cnt(S);
        for (int s = 0; ok && s < S; ++s) {
            const int q0 = stick_pw_ptr[s], q1 = stick_pw_ptr[s + 1];
            auto lsig = [&](int q) { return pw_z[q] <= n3 / 2 ? pw_z[q] : pw_z[q] - n3; };
            first[s] = pw_user[q0]; lmin[s] = lsig(q0); cnt[s] = q1 - q0;
            for (int q = q0 + 1; ok && q < q1; ++q) ok = pw_user[q] == pw_user[q - 1] + 1 && lsig(q) == lsig(q - 1) + 1;
        }
        if (ok) {
            run_tab.assign((size_t)T * kLinesPerTile * 4, 0);
            for (int tt = 0; tt < T; ++tt)
                for (int i = tile_ptr[tt]; i < tile_ptr[tt + 1]; ++i) {
                    const int s = tile_sticks[i];
                    int* e = &run_tab[((size_t)tt * kLinesPerTile + (i - tile_ptr[tt])) * 4];
                    e[0] = first[s]; e[1] = lmin[s]; e[2] = cnt[s];
                }
            runs_ok = (flags & VLOC_Z_BULK) ? 1 : 2;
        }
    }

    // ---- Gamma-point table for the z-passes that form and separate the
    // real band pairs themselves (used when every G and its -G share a tile):
    // per tile, {h, position of G, position of -G, 0} (position = z | line
    // << 16) for every half-list plane wave whose G lies in the tile
    std::vector<int> gamma_h_ptr, gamma_h;
    bool gamma_ok = false;
    if (flags & VLOC_GAMMA) {
        const int64_t nh = npw_user;
        std::vector<int> tile_of(npw, -1), pos_of(npw, 0);
        for (int tt = 0; tt < T; ++tt)
            for (int e = tile_pw_ptr[tt]; e < tile_pw_ptr[tt + 1]; ++e) {
                const int f = tile_pw[2 * e];
                tile_of[f] = tt;
                pos_of[f] = tile_pw[2 * e + 1];
            }
        gamma_ok = true;
        for (int64_t q = 0; gamma_ok && q < nh; ++q) gamma_ok = tile_of[q] == tile_of[gamma_neg[q]];
        if (gamma_ok) {
            std::vector<std::vector<int>> per(T);
            for (int64_t q = 0; q < nh; ++q) per[tile_of[q]].push_back((int)q);
            gamma_h_ptr.push_back(0);
            for (int tt = 0; tt < T; ++tt) {
                for (int q : per[tt]) gamma_h.insert(gamma_h.end(), {q, pos_of[q], pos_of[gamma_neg[q]], 0});
                gamma_h_ptr.push_back((int)(gamma_h.size() / 4));
            }
        }
    }

    // ---- host copy of the index tables, as the kernels read them
    {
        std::vector<int>& blob = p->host_tables;
        HostTableLayout& L = p->lay;
        auto append = [&](const std::vector<int>& v) { size_t off = blob.size(); blob.insert(blob.end(), v.begin(), v.end()); return off; };
        L.o_row = append(stick_row);
        L.o_tp = append(tile_ptr);
        L.o_ts = append(tile_sticks);
        L.o_tpp = append(tile_pw_ptr);
        if (blob.size() & 1) blob.push_back(0);  // int2 alignment of the entry list
        L.o_tpw = append(tile_pw);
        L.o_plp = append(plane_ptr);
        L.o_xr = append(xrow_plane);
        L.gok = gamma_ok ? 1 : 0;
        L.nh = (flags & VLOC_GAMMA) ? npw_user : 0;
        L.o_ghp = append(gamma_h_ptr);
        L.zd_rows = zd_rows;
        while (blob.size() & 3) blob.push_back(0);  // 16-byte alignment
        L.o_zd = append(zdense);
        L.zs = zs_ok;
        L.o_zs = append(zsh);
        L.runs = runs_ok;
        while (blob.size() & 3) blob.push_back(0);  // int4 alignment
        L.o_rn = append(run_tab);
        while (blob.size() & 3) blob.push_back(0);  // int4 alignment
        L.o_gh = append(gamma_h);
        L.total = blob.size();
        L.S = S; L.T = T; L.NP = NP;
        // the quarter-sphere x-plane pattern (x = 0..Q and n1 - Q .. n1 - 1,
        // Q = n1 / 4, planes in ascending x), which the x-pass kernels can
        // take at compile time; VLOC_NO_XQ (a test aid) turns the
        // specialisation off
        const int Q = n1 / 4;
        bool xq = NP == 2 * Q + 1 && Q >= 1 && std::getenv("VLOC_NO_XQ") == nullptr;
        for (int x = 0; xq && x < n1; ++x) {
            const int want = x <= Q ? x : x >= n1 - Q ? x - n1 + NP : -1;
            xq = xrow_plane[x] == want;
        }
        L.xq = xq ? 1 : 0;
        // every l within the quarter band of n3 (the z-pass kernels take the
        // band at compile time; VLOC_NO_XQ turns this off too)
        const int Q3 = n3 / 4;
        bool zq = Q3 >= 1 && std::getenv("VLOC_NO_XQ") == nullptr;
        for (int64_t q = 0; zq && q < npw; ++q) {
            const int z = pw_z[q];
            zq = z <= Q3 || z >= n3 - Q3;
        }
        L.zq = zq ? 1 : 0;
    }

    if (host_only) {
        p->chunk = 0;
        *out = p;
        return VLOC_OK;
    }
    // shared-memory budget of the largest kernel tile
    int dev = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev))) { free_plan(p); return cuda_fail(e, "cudaGetDevice"); }
    p->device = dev;
    int maxopt = 0;
    if ((e = cudaDeviceGetAttribute(&maxopt, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev))) {
        free_plan(p); return cuda_fail(e, "cudaDeviceGetAttribute");
    }
    if (smem_bytes_for(dbl, nmax) > (size_t)maxopt) { free_plan(p); return VLOC_ERR_SIZE; }
    p->smem_optin = maxopt;

    // ---- device tables (one allocation)
    cudaStream_t st = (cudaStream_t)stream;
    const std::vector<int>& blob = p->host_tables;
    if ((e = dmalloc((void**)&p->d_tables, blob.size() * sizeof(int)))) { free_plan(p); return cuda_fail(e, "cudaMalloc(tables)"); }
    if ((e = cudaMemcpyAsync(p->d_tables, blob.data(), blob.size() * sizeof(int), cudaMemcpyHostToDevice, st))) {
        free_plan(p); return cuda_fail(e, "upload tables");
    }
    p->dt = device_tables(p->d_tables, p->lay, n1, n2, n3, npw);
    // the pair-forming z-passes exist for the FP32 compile-time kernels;
    // VLOC_GAMMA_PACK (a test aid) keeps the separate pack / unpack passes
    p->gfused = p->gamma && p->lay.gok && !dbl && p->fast && has_ct(n3) && std::getenv("VLOC_GAMMA_PACK") == nullptr;

    // ---- twiddles exp(+2 pi i j / n), FP64-made
    for (int a = 0; a < 3; ++a) {
        if ((e = dmalloc((void**)&p->d_tw[a], (size_t)ns[a] * elem))) { free_plan(p); return cuda_fail(e, "cudaMalloc(twiddles)"); }
        if (launch_twiddles(dbl, p->d_tw[a], ns[a], st)) { free_plan(p); return cuda_fail(cudaGetLastError(), "twiddles"); }
    }
    if ((e = (cudaError_t)set_smem_limits(dbl, nmax, maxopt))) { free_plan(p); return cuda_fail(e, "cudaFuncSetAttribute"); }
    if ((e = dmalloc((void**)&p->d_err, sizeof(int)))) { free_plan(p); return cuda_fail(e, "cudaMalloc(error flag)"); }

    if ((e = cudaMemsetAsync(p->d_err, 0, sizeof(int), st))) { free_plan(p); return cuda_fail(e, "clear error flag"); }
    p->dt.err = p->d_err;
    if (p->df) {
        for (int a = 0; a < 3; ++a) {
            if ((e = dmalloc((void**)&p->d_twdf[a], (size_t)ns[a] * 32))) { free_plan(p); return cuda_fail(e, "cudaMalloc(df twiddles)"); }
            if (launch_twiddles_df(p->d_tw[a], p->d_twdf[a], ns[a], st)) { free_plan(p); return cuda_fail(cudaGetLastError(), "df twiddles"); }
        }
        if ((e = dmalloc((void**)&p->d_vdf, (size_t)N * 8))) { free_plan(p); return cuda_fail(e, "cudaMalloc(df V)"); }
    }

    // ---- workspace: cylinder [chunk][S][n3] + slab [chunk][NP][n2][n3]
    const size_t per_band = ((size_t)S * n3 + (size_t)NP * n2 * n3) * elem;
    long long chunk = max_bands_per_chunk;
    if (chunk <= 0) {
        // Enough bands per launch that every kernel runs many waves over the
        // 152 SMs (kernel tails and launch gaps dominate small chunks, which
        // measured slower even when their workspace stays in L2): a 6 GiB
        // workspace, at most a sixteenth of the free device memory, and at
        // most 2048 bands (small grids).  At 96^3 FP32 a 1024-band step is
        // then one chunk: 4.14 ms against 4.23 ms in 430-band chunks.
        size_t free_b = 0, total_b = 0;
        size_t target = (size_t)6 << 30;
        if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) target = std::min(target, free_b / 16);
        chunk = std::min<long long>(2048, std::max<long long>(1, (long long)(target / per_band)));
    }
    chunk = std::min<long long>(chunk, 65535);
    p->chunk = chunk;
    p->ws_bands = std::max<long long>(chunk, 2);
    p->ngroups = (int)((std::max<long long>(1, p->ws_bands / 2) + kGradBandsPerGroup - 1) / kGradBandsPerGroup);
    p->ws_bytes = per_band * (size_t)p->ws_bands + (size_t)N * sizeof(double) * (1 + p->ngroups);
    if ((e = dmalloc((void**)&p->d_cyl, (size_t)S * n3 * elem * p->ws_bands))) { free_plan(p); return cuda_fail(e, "cudaMalloc(cylinder)"); }
    if ((e = dmalloc((void**)&p->d_slab, (size_t)NP * n2 * n3 * elem * p->ws_bands))) { free_plan(p); return cuda_fail(e, "cudaMalloc(slab)"); }
    if (p->gamma) {
        if ((e = dmalloc((void**)&p->d_gamma_neg, sizeof(int) * (size_t)npw_user))) { free_plan(p); return cuda_fail(e, "cudaMalloc(gamma map)"); }
        if ((e = cudaMemcpyAsync(p->d_gamma_neg, gamma_neg.data(), sizeof(int) * (size_t)npw_user, cudaMemcpyHostToDevice, st))) {
            free_plan(p); return cuda_fail(e, "upload gamma map");
        }
        if ((e = dmalloc((void**)&p->d_gamma_buf, 2 * (size_t)p->chunk * npw * elem))) { free_plan(p); return cuda_fail(e, "cudaMalloc(gamma buffers)"); }
        p->ws_bytes += 2 * (size_t)p->chunk * npw * elem;
    }
    // tensor map over the slab workspace for the persistent TMA x-pass (FP32,
    // compile-time x length, even n3 so rows are 16-byte multiples)
    if ((flags & VLOC_X_TMA) && !dbl && p->fast && has_ct(n1) && (n3 % 2) == 0 && NP <= 256) {
        static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
        if (!encode) {
            cudaDriverEntryPointQueryResult q;
            void* fn = nullptr;
            if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                    cudaSuccess && q == cudaDriverEntryPointSuccess)
                encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
        }
        if (encode) {
            const cuuint64_t dims[4] = {(cuuint64_t)2 * n3, (cuuint64_t)n2, (cuuint64_t)NP, (cuuint64_t)p->ws_bands};
            const cuuint64_t strides[3] = {(cuuint64_t)n3 * 8, (cuuint64_t)n2 * n3 * 8, (cuuint64_t)NP * n2 * n3 * 8};
            const cuuint32_t box[4] = {64, 1, (cuuint32_t)NP, 1};
            const cuuint32_t estr[4] = {1, 1, 1, 1};
            if (encode(&p->k3tma.map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, p->d_slab, dims, strides, box, estr,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS) {
                p->k3tma.base = p->d_slab;
                p->k3tma.band_bytes = (size_t)NP * n2 * n3 * 8;
                p->k3tma.err = p->d_err;
                p->k3tma.skip_first = fault.tma_wait ? 1 : 0;
                p->k3tma_on = true;
            }
        }
    }

    // dL/dV accumulator [N] followed by the band groups' partial sums [ngroups][N]
    if ((e = dmalloc((void**)&p->d_acc, (size_t)N * sizeof(double) * (1 + p->ngroups)))) { free_plan(p); return cuda_fail(e, "cudaMalloc(acc)"); }
    if ((e = cudaStreamSynchronize(st))) { free_plan(p); return cuda_fail(e, "plan create sync"); }
    *out = p;
    return VLOC_OK;
}

int vloc_plan_set_schedule(vloc_plan p, int axis, int nst, const int32_t* radix) {
    if (!p || axis < 0 || axis > 2 || nst < 1 || nst > 4 || !radix) return VLOC_ERR_ARG;
    long long prod = 1;
    for (int i = 0; i < nst; ++i) {
        bool ok = false;
        for (int r : kRadices) ok = ok || r == radix[i];
        if (!ok) return VLOC_ERR_ARG;
        prod *= radix[i];
    }
    if (prod != p->ax.n[axis]) return VLOC_ERR_ARG;
    p->ax.nst[axis] = nst;
    for (int i = 0; i < 4; ++i) p->ax.radix[axis][i] = i < nst ? radix[i] : 0;
    p->fast = 0;
    p->df = false;
    p->k3tma_on = false;
    p->gfused = false;
    for (auto& g : p->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    p->graphs.clear();
    return VLOC_OK;
}

int vloc_plan_destroy(vloc_plan p) {
    if (!p) return VLOC_OK;
    if (p->flags & VLOC_HOST_ONLY) { delete p; return VLOC_OK; }
    cudaError_t e = cudaDeviceSynchronize();
    free_plan(p);
    return e == cudaSuccess ? VLOC_OK : cuda_fail(e, "destroy sync");
}

static bool aligned(const void* q, size_t a) { return ((uintptr_t)q % a) == 0; }
static bool overlap(const void* a, size_t na, const void* b, size_t nb) {
    const char *pa = (const char*)a, *pb = (const char*)b;
    return pa < pb + nb && pb < pa + na;
}

static int check_io(vloc_plan p, const void* c, const void* V, int64_t nb, const void* out) {
    if (!p || nb < 0) return VLOC_ERR_ARG;
    if (p->flags & VLOC_HOST_ONLY) return VLOC_ERR_STATE;
    if (nb == 0) return VLOC_OK;
    if (!c || !V || !out) return VLOC_ERR_ARG;
    const size_t re = p->dbl ? 8 : 4;
    if (!aligned(c, p->elem) || !aligned(out, p->elem) || !aligned(V, re)) return VLOC_ERR_ARG;
    const size_t bytes = (size_t)nb * p->npw_user * p->elem;
    if (c != out && overlap(c, bytes, out, bytes)) return VLOC_ERR_ARG;
    if (overlap(V, (size_t)p->N * re, out, bytes)) return VLOC_ERR_ARG;
    return VLOC_OK;
}

}  // extern "C"

// Launch one kernel of the chain, bracketed by timing events when profiling.
template <class F>
static int launch(vloc_plan p, int kind, cudaStream_t st, F&& f) {
    size_t i0 = 0;
    if (p->prof_on) {
        i0 = p->prof_recs.size() * 2;
        while (p->prof_pool.size() < i0 + 2) {
            cudaEvent_t e;
            cudaError_t err = cudaEventCreate(&e);
            if (err) return cuda_fail(err, "profiling event");
            p->prof_pool.push_back(e);
        }
        cudaEventRecord(p->prof_pool[i0], st);
    }
    const int rc = f();
    if (rc) return cuda_fail((cudaError_t)rc, "kernel launch");
    ++p->launches;
    if (p->prof_on) {
        cudaEventRecord(p->prof_pool[i0 + 1], st);
        p->prof_recs.push_back({kind, i0});
    }
    return VLOC_OK;
}

// VLOC_POISON_WORKSPACE (a test aid): fill the whole cylinder and slab
// workspace with all-ones bytes -- a NaN in FP32, FP64 and double-float --
// before each chunk, so that a pruned pass reading a cell no earlier pass of
// the chunk wrote makes the result non-finite.
static int poison(vloc_plan p, cudaStream_t st) {
    if (!p->poison) return VLOC_OK;
    const size_t cyl = (size_t)p->S * p->n3 * p->elem * p->ws_bands;
    const size_t slab = (size_t)p->NP * p->n2 * p->n3 * p->elem * p->ws_bands;
    cudaError_t e;
    if ((e = cudaMemsetAsync(p->d_cyl, 0xFF, cyl, st))) return cuda_fail(e, "poison cylinder");
    if ((e = cudaMemsetAsync(p->d_slab, 0xFF, slab, st))) return cuda_fail(e, "poison slab");
    return VLOC_OK;
}

extern "C" {

// out = A c over workspace chunks: K1, K2(+), K3, K2(-), K4 per chunk.
// With `diag` (device real [npw]) the gather adds diag * c: out = (diag + A) c.
static int apply_impl(vloc_plan p, const void* c, const void* V, int64_t nb, void* out, cudaStream_t st,
                      const void* diag = nullptr) {
    const size_t bstride = (size_t)p->npw * p->elem;
    const int dbl = p->dbl;
    const DevTables& t = p->dt;
    const LaunchAxes& ax = p->ax;
    if (p->df) {
        // double-float chain: its own twiddle tables, V as hi + lo pairs
        int rc;
        if ((rc = launch(p, KK_AUX, st, [&] { return launch_v_to_df(V, p->d_vdf, p->N, st); }))) return rc;
        for (int64_t b0 = 0; b0 < nb; b0 += p->chunk) {
            const long long cb = std::min<long long>(p->chunk, nb - b0);
            const void* cc = (const char*)c + b0 * bstride;
            void* oo = (char*)out + b0 * bstride;
            if ((rc = poison(p, st))) return rc;
            if ((rc = launch(p, KK_SCATTER_Z, st, [&] { return launch_k1_scatter_zpass(1, 2, t, ax, p->d_twdf[2], cc, cb, p->d_cyl, st); }))) return rc;
            if ((rc = launch(p, KK_Y_INV, st, [&] { return launch_k2_ypass(1, 2, +1, t, ax, p->d_twdf[1], cb, p->d_cyl, p->d_slab, st); }))) return rc;
            if ((rc = launch(p, KK_X_V, st, [&] { return launch_k3_xpass_v(1, 2, t, ax, p->d_twdf[0], p->d_vdf, cb, p->d_slab, st); }))) return rc;
            if ((rc = launch(p, KK_Y_FWD, st, [&] { return launch_k2_ypass(1, 2, -1, t, ax, p->d_twdf[1], cb, p->d_cyl, p->d_slab, st); }))) return rc;
            if ((rc = launch(p, KK_Z_GATHER, st, [&] { return launch_k4_zpass_gather(1, 2, t, ax, p->d_twdf[2], p->d_cyl, cb, oo, diag, cc, st); }))) return rc;
        }
        return VLOC_OK;
    }
    for (int64_t b0 = 0; b0 < nb; b0 += p->chunk) {
        const long long cb = std::min<long long>(p->chunk, nb - b0);
        const void* cc = (const char*)c + b0 * bstride;
        void* oo = (char*)out + b0 * bstride;
        int rc;
        if ((rc = poison(p, st))) return rc;
        if ((rc = launch(p, KK_SCATTER_Z, st, [&] { return launch_k1_scatter_zpass(dbl, p->fast, t, ax, p->d_tw[2], cc, cb, p->d_cyl, st); }))) return rc;
        if ((rc = launch(p, KK_Y_INV, st, [&] { return launch_k2_ypass(dbl, p->fast, +1, t, ax, p->d_tw[1], cb, p->d_cyl, p->d_slab, st); }))) return rc;
        if ((rc = launch(p, KK_X_V, st, [&] { return launch_k3_xpass_v(dbl, p->fast, t, ax, p->d_tw[0], V, cb, p->d_slab, st, p->k3tma_on ? &p->k3tma : nullptr); }))) return rc;
        if ((rc = launch(p, KK_Y_FWD, st, [&] { return launch_k2_ypass(dbl, p->fast, -1, t, ax, p->d_tw[1], cb, p->d_cyl, p->d_slab, st); }))) return rc;
        if ((rc = launch(p, KK_Z_GATHER, st, [&] { return launch_k4_zpass_gather(dbl, p->fast, t, ax, p->d_tw[2], p->d_cyl, cb, oo, diag, cc, st); }))) return rc;
    }
    return VLOC_OK;
}

}  // extern "C"

// Gamma-point real mode: bands 2p and 2p+1 (real in r-space) travel as one
// complex band a + i b through the chain; each result pair is separated with
// U(G) and conj U(-G).
// Gamma-point apply with the pairs formed and separated inside the z-passes
// (FP32 compile-time kernels, every G in the same tile as its -G): no pack
// or unpack pass and no pair buffers.
static int gamma_apply_fused(vloc_plan p, const void* c, const void* V, int64_t nb, void* out, cudaStream_t st,
                             const void* diag) {
    const long long npairs = (nb + 1) / 2;
    const size_t ustride = (size_t)p->npw_user * p->elem;
    const DevTables& t = p->dt;
    const LaunchAxes& ax = p->ax;
    for (long long p0 = 0; p0 < npairs; p0 += p->chunk) {
        const long long cp = std::min<long long>(p->chunk, npairs - p0);
        const long long b0 = 2 * p0, bn = std::min<long long>(nb - b0, 2 * cp);
        const void* cc = (const char*)c + b0 * ustride;
        void* oo = (char*)out + b0 * ustride;
        int rc;
        if ((rc = poison(p, st))) return rc;
        if ((rc = launch(p, KK_SCATTER_Z, st, [&] { return launch_k1_gamma(t, p->d_tw[2], cc, cp, bn, p->d_cyl, st); }))) return rc;
        if ((rc = launch(p, KK_Y_INV, st, [&] { return launch_k2_ypass(0, p->fast, +1, t, ax, p->d_tw[1], cp, p->d_cyl, p->d_slab, st); }))) return rc;
        if ((rc = launch(p, KK_X_V, st, [&] { return launch_k3_xpass_v(0, p->fast, t, ax, p->d_tw[0], V, cp, p->d_slab, st, p->k3tma_on ? &p->k3tma : nullptr); }))) return rc;
        if ((rc = launch(p, KK_Y_FWD, st, [&] { return launch_k2_ypass(0, p->fast, -1, t, ax, p->d_tw[1], cp, p->d_cyl, p->d_slab, st); }))) return rc;
        if ((rc = launch(p, KK_Z_GATHER, st, [&] { return launch_k4_gamma(t, p->d_tw[2], p->d_cyl, cp, bn, oo, diag, cc, st); }))) return rc;
    }
    return VLOC_OK;
}

static int gamma_apply(vloc_plan p, const void* c, const void* V, int64_t nb, void* out, cudaStream_t st,
                       const void* diag) {
    if (p->gfused) return gamma_apply_fused(p, c, V, nb, out, st, diag);
    const long long npairs = (nb + 1) / 2;
    const size_t full = (size_t)p->npw * p->elem;
    char* C = (char*)p->d_gamma_buf;
    char* U = C + (size_t)p->chunk * full;
    for (long long p0 = 0; p0 < npairs; p0 += p->chunk) {
        const long long cp = std::min<long long>(p->chunk, npairs - p0);
        const long long b0 = 2 * p0, bn = std::min<long long>(nb - b0, 2 * cp);
        const size_t ustride = (size_t)p->npw_user * p->elem;
        int rc;
        if ((rc = launch(p, KK_GAMMA, st, [&] {
                 return launch_gamma_pack(p->dbl, (const char*)c + b0 * ustride, bn, p->npw_user, p->d_gamma_neg,
                                          p->npw, C, cp, st);
             })))
            return rc;
        if ((rc = apply_impl(p, C, V, cp, U, st))) return rc;
        if ((rc = launch(p, KK_GAMMA, st, [&] {
                 return launch_gamma_unpack(p->dbl, U, cp, p->npw, p->d_gamma_neg, p->npw_user, (char*)out + b0 * ustride,
                                            bn, diag, (const char*)c + b0 * ustride, st);
             })))
            return rc;
    }
    return VLOC_OK;
}

static int apply_any(vloc_plan p, const void* c, const void* V, int64_t nb, void* out, cudaStream_t st,
                     const void* diag = nullptr) {
    return p->gamma ? gamma_apply(p, c, V, nb, out, st, diag) : apply_impl(p, c, V, nb, out, st, diag);
}

// Replay (or capture, then replay) the work `enqueue` puts on a stream as one
// CUDA graph, cached in `owner` under `key`; `plans` are the plans whose
// kernels the work launches.  Captured on the owner's private stream, then
// launched on `st`, so it stays ordered with the caller's work.
template <class F>
static int graph_run(vloc_plan owner, const std::vector<vloc_plan>& plans, std::vector<uintptr_t> key,
                     cudaStream_t st, F&& enqueue) {
    cudaError_t e;
    for (auto& g : owner->graphs)
        if (g.key == key) {
            g.last_use = ++owner->use_clock;
            if ((e = cudaGraphLaunch(g.exec, st))) return cuda_fail(e, "cudaGraphLaunch");
            for (auto& k : g.kernels) k.first->launches += k.second;
            return VLOC_OK;
        }
    if (!owner->cap_stream && (e = cudaStreamCreateWithFlags(&owner->cap_stream, cudaStreamNonBlocking)))
        return cuda_fail(e, "capture stream");
    std::vector<long long> l0;
    std::vector<bool> prof;
    for (vloc_plan q : plans) {
        l0.push_back(q->launches);
        prof.push_back(q->prof_on);
        q->prof_on = false;  // no timing events inside a graph
    }
    auto restore = [&] {
        for (size_t i = 0; i < plans.size(); ++i) plans[i]->prof_on = prof[i];
    };
    if ((e = cudaStreamBeginCapture(owner->cap_stream, cudaStreamCaptureModeThreadLocal))) {
        restore();
        return cuda_fail(e, "cudaStreamBeginCapture");
    }
    const int rc = enqueue(owner->cap_stream);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(owner->cap_stream, &graph);
    restore();
    vloc_plan_s::GraphEntry ent;
    for (size_t i = 0; i < plans.size(); ++i) {
        ent.kernels.push_back({plans[i], plans[i]->launches - l0[i]});
        plans[i]->launches = l0[i];
    }
    if (rc || e) {
        if (graph) cudaGraphDestroy(graph);
        return rc ? rc : cuda_fail(e, "cudaStreamEndCapture");
    }
    e = cudaGraphInstantiate(&ent.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e) return cuda_fail(e, "cudaGraphInstantiate");
    if (owner->graphs.size() >= 8) {  // least recently used out
        auto it = std::min_element(owner->graphs.begin(), owner->graphs.end(),
                                   [](const auto& a, const auto& b) { return a.last_use < b.last_use; });
        cudaGraphExecDestroy(it->exec);
        owner->graphs.erase(it);
    }
    ent.key = std::move(key);
    ent.last_use = ++owner->use_clock;
    owner->graphs.push_back(std::move(ent));
    auto& g = owner->graphs.back();
    if ((e = cudaGraphLaunch(g.exec, st))) return cuda_fail(e, "cudaGraphLaunch");
    for (auto& k : g.kernels) k.first->launches += k.second;
    return VLOC_OK;
}

extern "C" {

int vloc_apply(vloc_plan p, const void* c, const void* V, int64_t nb, void* out, void* stream) {
    int rc = check_io(p, c, V, nb, out);
    if (rc || nb == 0) return rc;
    if (p->flags & VLOC_GRAPH)
        return graph_run(p, {p}, {(uintptr_t)c, (uintptr_t)V, (uintptr_t)nb, (uintptr_t)out}, (cudaStream_t)stream,
                         [&](cudaStream_t cs) { return apply_any(p, c, V, nb, out, cs); });
    return apply_any(p, c, V, nb, out, (cudaStream_t)stream);
}

int vloc_apply_h(vloc_plan p, const void* c, const void* V, const void* diag, int64_t nb, void* out, void* stream) {
    int rc = check_io(p, c, V, nb, out);
    if (rc || nb == 0) return rc;
    if (!diag) return vloc_apply(p, c, V, nb, out, stream);
    const size_t re = p->dbl ? 8 : 4;
    if (!aligned(diag, re)) return VLOC_ERR_ARG;
    if (overlap(diag, (size_t)p->npw_user * re, out, (size_t)nb * p->npw_user * p->elem)) return VLOC_ERR_ARG;
    if (p->flags & VLOC_GRAPH)
        return graph_run(p, {p}, {(uintptr_t)c, (uintptr_t)V, (uintptr_t)nb, (uintptr_t)out, (uintptr_t)diag},
                         (cudaStream_t)stream, [&](cudaStream_t cs) { return apply_any(p, c, V, nb, out, cs, diag); });
    return apply_any(p, c, V, nb, out, (cudaStream_t)stream, diag);
}

int vloc_apply_adjoint(vloc_plan p, const void* c, const void* V, int64_t nb, void* out, void* stream) {
    // A^H = (1/N) S^T F- diag(conj V) F+ S = A for real V.
    return vloc_apply(p, c, V, nb, out, stream);
}

int vloc_backward(vloc_plan p, const void* c, const void* gout, const void* V, int64_t nb, void* gc, void* gV,
                  void* stream) {
    if (!p || nb < 0) return VLOC_ERR_ARG;
    if ((p->flags & VLOC_HOST_ONLY) || p->gamma) return VLOC_ERR_STATE;
    if (!gc && !gV) return VLOC_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t re = p->dbl ? 8 : 4;
    const size_t bytes = (size_t)nb * p->npw * p->elem;
    if (gc) {
        int rc = check_io(p, gout, V, nb, gc);
        if (rc) return rc;
        if (c && nb > 0 && overlap(c, bytes, gc, bytes)) return VLOC_ERR_ARG;
    }
    if (gV) {
        if (!aligned(gV, re) || (nb > 0 && (!c || !gout || !V))) return VLOC_ERR_ARG;
        if (nb > 0 && (!aligned(c, p->elem) || !aligned(gout, p->elem))) return VLOC_ERR_ARG;
        if (nb > 0 && (overlap(gV, (size_t)p->N * re, c, bytes) || overlap(gV, (size_t)p->N * re, gout, bytes)))
            return VLOC_ERR_ARG;
        if (gc && overlap(gV, (size_t)p->N * re, gc, bytes)) return VLOC_ERR_ARG;
        const int dbl = p->dbl;
        const DevTables& t = p->dt;
        const LaunchAxes& ax = p->ax;
        if (grad_smem_bytes(dbl, p->n1) > (size_t)p->smem_optin) return VLOC_ERR_SIZE;
        int rc;
        if ((rc = launch(p, KK_AUX, st, [&] { return launch_zero_f64(p->d_acc, p->N, st); }))) return rc;
        const long long half = std::max<long long>(1, p->ws_bands / 2);
        const size_t cyl_band = (size_t)p->S * p->n3 * p->elem;
        const size_t slab_band = (size_t)p->NP * p->n2 * p->n3 * p->elem;
        char* cylC = (char*)p->d_cyl;
        char* cylG = cylC + half * cyl_band;
        char* slabC = (char*)p->d_slab;
        char* slabG = slabC + half * slab_band;
        const size_t bstride = (size_t)p->npw * p->elem;
        for (int64_t b0 = 0; b0 < nb; b0 += half) {
            const long long cb = std::min<long long>(half, nb - b0);
            const void* cc = (const char*)c + b0 * bstride;
            const void* gg = (const char*)gout + b0 * bstride;
            if ((rc = poison(p, st))) return rc;
            if ((rc = launch(p, KK_SCATTER_Z, st, [&] { return launch_k1_scatter_zpass(dbl, p->fast, t, ax, p->d_tw[2], cc, cb, cylC, st); }))) return rc;
            if ((rc = launch(p, KK_Y_INV, st, [&] { return launch_k2_ypass(dbl, p->fast, +1, t, ax, p->d_tw[1], cb, cylC, slabC, st); }))) return rc;
            if ((rc = launch(p, KK_SCATTER_Z, st, [&] { return launch_k1_scatter_zpass(dbl, p->fast, t, ax, p->d_tw[2], gg, cb, cylG, st); }))) return rc;
            if ((rc = launch(p, KK_Y_INV, st, [&] { return launch_k2_ypass(dbl, p->fast, +1, t, ax, p->d_tw[1], cb, cylG, slabG, st); }))) return rc;
            int used = 1;
            double* partial = p->d_acc + p->N;
            if ((rc = launch(p, KK_GRAD_V, st, [&] { return launch_k3b_grad_v(dbl, p->fast, t, ax, p->d_tw[0], slabC, slabG, cb, (int)kGradBandsPerGroup, partial, &used, st); }))) return rc;
            if ((rc = launch(p, KK_AUX, st, [&] { return launch_reduce_partials(partial, used, p->N, p->d_acc, st); }))) return rc;
            if (gc) {
                // dL/dc = A g continues from g's slab (its z- and y-passes are
                // already done): x-pass with V, forward y-pass, z-pass + gather
                void* gg_out = (char*)gc + b0 * bstride;
                if ((rc = launch(p, KK_X_V, st, [&] { return launch_k3_xpass_v(dbl, p->fast, t, ax, p->d_tw[0], V, cb, slabG, st, p->k3tma_on ? &p->k3tma : nullptr); }))) return rc;
                if ((rc = launch(p, KK_Y_FWD, st, [&] { return launch_k2_ypass(dbl, p->fast, -1, t, ax, p->d_tw[1], cb, cylG, slabG, st); }))) return rc;
                if ((rc = launch(p, KK_Z_GATHER, st, [&] { return launch_k4_zpass_gather(dbl, p->fast, t, ax, p->d_tw[2], cylG, cb, gg_out, nullptr, nullptr, st); }))) return rc;
            }
        }
        if ((rc = launch(p, KK_AUX, st, [&] { return launch_finish_grad_v(dbl, p->d_acc, gV, p->N, st); }))) return rc;
        return VLOC_OK;
    }
    if (gc && nb > 0) {
        int rc = apply_impl(p, gout, V, nb, gc, st);
        if (rc) return rc;
    }
    return VLOC_OK;
}

// ---- the two halves of the chain on their own, and the charge density
int vloc_to_real(vloc_plan p, const void* c, int64_t nb, void* psi, void* stream) {
    if (!p || nb < 0) return VLOC_ERR_ARG;
    if ((p->flags & VLOC_HOST_ONLY) || p->gamma) return VLOC_ERR_STATE;
    if (nb == 0) return VLOC_OK;
    if (!c || !psi || !aligned(c, p->elem) || !aligned(psi, p->elem)) return VLOC_ERR_ARG;
    const size_t bstride = (size_t)p->npw * p->elem, gstride = (size_t)p->N * p->elem;
    if (overlap(c, nb * bstride, psi, nb * gstride)) return VLOC_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int dbl = p->dbl;
    const DevTables& t = p->dt;
    const LaunchAxes& ax = p->ax;
    for (int64_t b0 = 0; b0 < nb; b0 += p->chunk) {
        const long long cb = std::min<long long>(p->chunk, nb - b0);
        const void* cc = (const char*)c + b0 * bstride;
        void* gg = (char*)psi + b0 * gstride;
        int rc;
        if ((rc = poison(p, st))) return rc;
        if ((rc = launch(p, KK_SCATTER_Z, st, [&] { return launch_k1_scatter_zpass(dbl, p->fast, t, ax, p->d_tw[2], cc, cb, p->d_cyl, st); }))) return rc;
        if ((rc = launch(p, KK_Y_INV, st, [&] { return launch_k2_ypass(dbl, p->fast, +1, t, ax, p->d_tw[1], cb, p->d_cyl, p->d_slab, st); }))) return rc;
        if ((rc = launch(p, KK_X_TO_GRID, st, [&] { return launch_k3_grid(dbl, p->fast, +1, t, ax, p->d_tw[0], cb, p->d_slab, gg, st); }))) return rc;
    }
    return VLOC_OK;
}

int vloc_to_recip(vloc_plan p, const void* u, int64_t nb, void* out, void* stream) {
    if (!p || nb < 0) return VLOC_ERR_ARG;
    if ((p->flags & VLOC_HOST_ONLY) || p->gamma) return VLOC_ERR_STATE;
    if (nb == 0) return VLOC_OK;
    if (!u || !out || !aligned(u, p->elem) || !aligned(out, p->elem)) return VLOC_ERR_ARG;
    const size_t bstride = (size_t)p->npw * p->elem, gstride = (size_t)p->N * p->elem;
    if (overlap(u, nb * gstride, out, nb * bstride)) return VLOC_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int dbl = p->dbl;
    const DevTables& t = p->dt;
    const LaunchAxes& ax = p->ax;
    for (int64_t b0 = 0; b0 < nb; b0 += p->chunk) {
        const long long cb = std::min<long long>(p->chunk, nb - b0);
        void* gg = (char*)const_cast<void*>(u) + b0 * gstride;
        void* oo = (char*)out + b0 * bstride;
        int rc;
        if ((rc = poison(p, st))) return rc;
        if ((rc = launch(p, KK_X_FROM_GRID, st, [&] { return launch_k3_grid(dbl, p->fast, -1, t, ax, p->d_tw[0], cb, p->d_slab, gg, st); }))) return rc;
        if ((rc = launch(p, KK_Y_FWD, st, [&] { return launch_k2_ypass(dbl, p->fast, -1, t, ax, p->d_tw[1], cb, p->d_cyl, p->d_slab, st); }))) return rc;
        if ((rc = launch(p, KK_Z_GATHER, st, [&] { return launch_k4_zpass_gather(dbl, p->fast, t, ax, p->d_tw[2], p->d_cyl, cb, oo, nullptr, nullptr, st); }))) return rc;
    }
    return VLOC_OK;
}

int vloc_density(vloc_plan p, const void* c, const void* occ, int64_t nb, void* rho, void* stream) {
    if (!p || nb < 0 || !rho) return VLOC_ERR_ARG;
    if (p->flags & VLOC_HOST_ONLY) return VLOC_ERR_STATE;
    const size_t re = p->dbl ? 8 : 4;
    const size_t ustride = (size_t)p->npw_user * p->elem;
    if (!aligned(rho, re) || (occ && !aligned(occ, re))) return VLOC_ERR_ARG;
    if (nb > 0 && (!c || !aligned(c, p->elem))) return VLOC_ERR_ARG;
    if (nb > 0 && overlap(rho, (size_t)p->N * re, c, nb * ustride)) return VLOC_ERR_ARG;
    if (nb > 0 && occ && overlap(rho, (size_t)p->N * re, occ, nb * re)) return VLOC_ERR_ARG;
    if (density_smem_bytes(p->dbl, p->n1) > (size_t)p->smem_optin) return VLOC_ERR_SIZE;
    cudaStream_t st = (cudaStream_t)stream;
    const int dbl = p->dbl;
    const DevTables& t = p->dt;
    const LaunchAxes& ax = p->ax;
    int rc;
    const size_t slab_band = (size_t)p->NP * p->n2 * p->n3 * p->elem;
    // bands per density x-pass: the partial buffer holds ngroups FP64 grids,
    // or twice as many FP32 ones
    const int pf32 = density_partials_f32(dbl, p->fast, t);
    const long long per_pass = (long long)p->ngroups * (pf32 ? 2 : 1) * kGradBandsPerGroup;
    double* partial = p->d_acc + p->N;
    // FP32 partials: the first reduction starts the FP64 accumulator and the
    // last writes rho itself, so no zeroing and no finishing pass
    const bool fused = pf32 && nb > 0;
    bool first = true;
    if (!fused && (rc = launch(p, KK_AUX, st, [&] { return launch_zero_f64(p->d_acc, p->N, st); }))) return rc;
    // K1 + K2 on `cb` complex bands at `src` (stride npw), then the density
    // x-pass; `base` is the global index of the chunk's first (pair) band,
    // `last` says that no chunk follows.
    auto chunk_density = [&](const void* src, long long cb, long long base, int pair, bool last) -> int {
        int r;
        if ((r = poison(p, st))) return r;
        if ((r = launch(p, KK_SCATTER_Z, st, [&] { return launch_k1_scatter_zpass(dbl, p->fast, t, ax, p->d_tw[2], src, cb, p->d_cyl, st); }))) return r;
        if ((r = launch(p, KK_Y_INV, st, [&] { return launch_k2_ypass(dbl, p->fast, +1, t, ax, p->d_tw[1], cb, p->d_cyl, p->d_slab, st); }))) return r;
        for (long long j0 = 0; j0 < cb; j0 += per_pass) {
            const long long m = std::min(per_pass, cb - j0);
            int used = 1;
            const void* sl = (const char*)p->d_slab + j0 * slab_band;
            if ((r = launch(p, KK_DENSITY, st, [&] {
                     return launch_k3d_density(dbl, p->fast, t, ax, p->d_tw[0], sl, m, (int)kGradBandsPerGroup, occ,
                                               base + j0, pair, nb, partial, &used, st);
                 })))
                return r;
            const bool fin = last && j0 + m >= cb;
            if ((r = launch(p, KK_AUX, st, [&] {
                     return pf32 ? launch_reduce_partials_f32((const float*)partial, used, p->N, p->d_acc, first,
                                                              fin ? (float*)rho : nullptr, st)
                                 : launch_reduce_partials(partial, used, p->N, p->d_acc, st);
                 })))
                return r;
            first = false;
        }
        return VLOC_OK;
    };
    if (!p->gamma) {
        for (int64_t b0 = 0; b0 < nb; b0 += p->chunk) {
            const long long cb = std::min<long long>(p->chunk, nb - b0);
            if ((rc = chunk_density((const char*)c + b0 * ustride, cb, b0, 0, b0 + cb >= nb))) return rc;
        }
    } else {
        // Gamma-point pairs: psi_2p + i psi_2p+1, both real, so |.|^2 splits
        // into the two bands' squares on the real and imaginary parts
        const long long npairs = (nb + 1) / 2;
        for (long long p0 = 0; p0 < npairs; p0 += p->chunk) {
            const long long cp = std::min<long long>(p->chunk, npairs - p0);
            const long long bn = std::min<long long>(nb - 2 * p0, 2 * cp);
            if ((rc = launch(p, KK_GAMMA, st, [&] {
                     return launch_gamma_pack(dbl, (const char*)c + 2 * p0 * ustride, bn, p->npw_user, p->d_gamma_neg,
                                              p->npw, p->d_gamma_buf, cp, st);
                 })))
                return rc;
            if ((rc = chunk_density(p->d_gamma_buf, cp, p0, 1, p0 + cp >= npairs))) return rc;
        }
    }
    if (fused) return VLOC_OK;
    return launch(p, KK_AUX, st, [&] { return launch_finish_grad_v(dbl, p->d_acc, rho, p->N, st); });
}

int vloc_apply_batched(int ninst, const vloc_plan* plans, const void* const* c, const void* const* V,
                       const int64_t* nb, void* const* out, void* stream) {
    if (ninst < 0 || (ninst > 0 && (!plans || !c || !V || !nb || !out))) return VLOC_ERR_ARG;
    for (int i = 0; i < ninst; ++i) {
        if (!plans[i] || plans[i]->dbl != plans[0]->dbl) return VLOC_ERR_ARG;
        int rc = check_io(plans[i], c[i], V[i], nb[i], out[i]);
        if (rc) return rc;
    }
    auto enqueue = [&](cudaStream_t cs) {
        for (int i = 0; i < ninst; ++i) {
            if (nb[i] == 0) continue;
            int rc = apply_any(plans[i], c[i], V[i], nb[i], out[i], cs);
            if (rc) return rc;
        }
        return (int)VLOC_OK;
    };
    bool all_graph = ninst > 0;
    for (int i = 0; i < ninst; ++i) all_graph = all_graph && (plans[i]->flags & VLOC_GRAPH);
    if (!all_graph) return enqueue((cudaStream_t)stream);
    // Captured as parallel branches: instance i runs on branch (i mod K) so
    // independent instances (each with its own workspace) overlap and fill
    // one another's kernel tails; instances sharing a plan share a branch.
    vloc_plan owner = plans[0];
    const int K = std::min(ninst, (int)kBatchBranches);
    cudaError_t e;
    while ((int)owner->branch_streams.size() < K) {
        cudaStream_t s;
        if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking))) return cuda_fail(e, "branch stream");
        owner->branch_streams.push_back(s);
        cudaEvent_t ev;
        if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming))) return cuda_fail(e, "branch event");
        owner->branch_events.push_back(ev);
    }
    if (!owner->fork_event && (e = cudaEventCreateWithFlags(&owner->fork_event, cudaEventDisableTiming)))
        return cuda_fail(e, "fork event");
    auto branched = [&](cudaStream_t cs) {
        cudaError_t er;
        if ((er = cudaEventRecord(owner->fork_event, cs))) return cuda_fail(er, "fork");
        std::vector<int> branch_of(ninst);
        for (int i = 0; i < ninst; ++i) {
            branch_of[i] = i % K;
            for (int j = 0; j < i; ++j)
                if (plans[j] == plans[i]) { branch_of[i] = branch_of[j]; break; }
        }
        for (int b = 0; b < K; ++b)
            if ((er = cudaStreamWaitEvent(owner->branch_streams[b], owner->fork_event, 0))) return cuda_fail(er, "fork wait");
        for (int i = 0; i < ninst; ++i) {
            if (nb[i] == 0) continue;
            int rc = apply_any(plans[i], c[i], V[i], nb[i], out[i], owner->branch_streams[branch_of[i]]);
            if (rc) return rc;
        }
        for (int b = 0; b < K; ++b) {
            if ((er = cudaEventRecord(owner->branch_events[b], owner->branch_streams[b]))) return cuda_fail(er, "join");
            if ((er = cudaStreamWaitEvent(cs, owner->branch_events[b], 0))) return cuda_fail(er, "join wait");
        }
        return (int)VLOC_OK;
    };
    // the whole batch as one graph launch, cached on the first plan
    std::vector<uintptr_t> key{(uintptr_t)ninst};
    std::vector<vloc_plan> ps;
    for (int i = 0; i < ninst; ++i) {
        key.insert(key.end(), {(uintptr_t)plans[i], (uintptr_t)c[i], (uintptr_t)V[i], (uintptr_t)nb[i], (uintptr_t)out[i]});
        if (std::find(ps.begin(), ps.end(), plans[i]) == ps.end()) ps.push_back(plans[i]);
    }
    return graph_run(plans[0], ps, std::move(key), (cudaStream_t)stream, branched);
}

// Host-buffer apply; `blocking`: synchronise before return, otherwise leave
// the caller's stream waiting for the last copy out, with the staging slots'
// state kept for the next call (consecutive calls then overlap one call's
// last copies with the next call's first ones).
static int apply_host_impl(vloc_plan p, const void* ch, const void* Vh, int64_t nb, void* oh, void* stream,
                           bool blocking) {
    if (!p || nb < 0) return VLOC_ERR_ARG;
    if ((p->flags & VLOC_HOST_ONLY) || p->gamma) return VLOC_ERR_STATE;
    if (nb == 0) return VLOC_OK;
    if (!ch || !Vh || !oh) return VLOC_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lock(p->mu);
    const size_t re = p->dbl ? 8 : 4;
    const size_t bstride = (size_t)p->npw * p->elem;
    // staging chunks: at most 256 bands, so copies in, compute and copies
    // out of neighbouring chunks overlap (H2D and D2H on separate streams)
    const long long sb = std::min<long long>(p->chunk, VLOC_STAGE_BANDS);
    const size_t vbytes = (size_t)p->N * re;
    auto align = [](size_t x) { return (x + 255) & ~(size_t)255; };
    constexpr int K = VLOC_STAGE_SLOTS;
    static_assert(K >= 2 && K <= 4, "staging slots");
    const size_t need = align(vbytes) + 2 * K * align((size_t)sb * bstride);
    cudaError_t e;
    if (p->stage_bytes < need) {
        cudaFree(p->d_stage);
        p->d_stage = nullptr;
        p->stage_bytes = 0;
        if ((e = cudaMalloc(&p->d_stage, need))) return cuda_fail(e, "cudaMalloc(staging)");
        p->stage_bytes = need;
        for (bool& u : p->stage_used) u = false;  // fresh slots (cudaFree waited for the old ones)
        p->stage_next = 0;
        if (!p->copy_stream && (e = cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking)))
            return cuda_fail(e, "copy stream");
        if (!p->d2h_stream && (e = cudaStreamCreateWithFlags(&p->d2h_stream, cudaStreamNonBlocking)))
            return cuda_fail(e, "copy stream");
        for (auto& ev : p->ev)
            if (!ev && (e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming))) return cuda_fail(e, "events");
    }
    char* base = (char*)p->d_stage;
    char* dV = base;
    char* slot_in[K];
    char* slot_out[K];
    size_t off = align(vbytes);
    for (int s = 0; s < K; ++s) {
        slot_in[s] = base + off; off += align((size_t)sb * bstride);
        slot_out[s] = base + off; off += align((size_t)sb * bstride);
    }
    if ((e = cudaMemcpyAsync(dV, Vh, vbytes, cudaMemcpyHostToDevice, st))) return cuda_fail(e, "H2D V");
    // Chunk sizes: ramps growing by VLOC_STAGE_RAMP / 2 from 32 bands at both
    // ends (while they fit around one full chunk), so the first copy in and
    // the last copy out, which nothing overlaps, are short; chunks of at most
    // sb bands in between.  Measured on GB300 (96^3, 1024 bands): doubling
    // ramps and a 192-256 band middle beat fixed 256-band chunks by 8%.
    std::vector<long long> sizes;
    {
        std::vector<long long> front;
        long long rest = nb;
        for (long long r = 32; VLOC_STAGE_RAMP > 2 && r < sb; r = (r * VLOC_STAGE_RAMP / 2 + 7) / 8 * 8)
            if (rest >= 2 * r + sb) { front.push_back(r); rest -= 2 * r; }
        sizes = front;
        // the middle split evenly (a short chunk right after a full one would
        // stall on the full one's copy out)
        const long long m = (rest + sb - 1) / sb;
        for (long long k = 0; k < m; ++k) sizes.push_back(rest * (k + 1) / m - rest * k / m);
        sizes.insert(sizes.end(), front.rbegin(), front.rend());
    }
    // per slot s: ev[s] input copied in, ev[K+s] result computed, ev[2K+s]
    // result copied out.  A slot's input is overwritten only after the chunk
    // K back has been computed, its output only after that chunk's result
    // has been copied out.
    const int64_t nchunks = (int64_t)sizes.size();
    int64_t b0 = 0;
    for (int64_t i = 0; i < nchunks; b0 += sizes[i], ++i) {
        const int s = (int)((p->stage_next + i) % K);
        const long long cb = sizes[i];
        const bool used = p->stage_used[s];  // an earlier chunk (of this or an earlier call) used the slot
        if (used && (e = cudaStreamWaitEvent(p->copy_stream, p->ev[K + s], 0))) return cuda_fail(e, "wait");
        if ((e = cudaMemcpyAsync(slot_in[s], (const char*)ch + b0 * bstride, cb * bstride, cudaMemcpyHostToDevice, p->copy_stream)))
            return cuda_fail(e, "H2D coeffs");
        if ((e = cudaEventRecord(p->ev[s], p->copy_stream))) return cuda_fail(e, "record");
        if ((e = cudaStreamWaitEvent(st, p->ev[s], 0))) return cuda_fail(e, "wait");
        if (used && (e = cudaStreamWaitEvent(st, p->ev[2 * K + s], 0))) return cuda_fail(e, "wait");
        int rc = apply_impl(p, slot_in[s], dV, cb, slot_out[s], st);
        if (rc) return rc;
        if ((e = cudaEventRecord(p->ev[K + s], st))) return cuda_fail(e, "record");
        if ((e = cudaStreamWaitEvent(p->d2h_stream, p->ev[K + s], 0))) return cuda_fail(e, "wait");
        if ((e = cudaMemcpyAsync((char*)oh + b0 * bstride, slot_out[s], cb * bstride, cudaMemcpyDeviceToHost, p->d2h_stream)))
            return cuda_fail(e, "D2H out");
        if ((e = cudaEventRecord(p->ev[2 * K + s], p->d2h_stream))) return cuda_fail(e, "record");
        p->stage_used[s] = true;
    }
    p->stage_next = (int)((p->stage_next + nchunks) % K);
    if (!blocking) {
        // the caller's stream reaches this point once every result is in host memory
        const int last = (int)((p->stage_next + K - 1) % K);
        if ((e = cudaStreamWaitEvent(st, p->ev[2 * K + last], 0))) return cuda_fail(e, "wait copy out");
        return VLOC_OK;
    }
    if ((e = cudaStreamSynchronize(p->d2h_stream))) return cuda_fail(e, "sync copy");
    if ((e = cudaStreamSynchronize(p->copy_stream))) return cuda_fail(e, "sync copy");
    if ((e = cudaStreamSynchronize(st))) return cuda_fail(e, "sync");
    return VLOC_OK;
}

int vloc_apply_host(vloc_plan p, const void* ch, const void* Vh, int64_t nb, void* oh, void* stream) {
    return apply_host_impl(p, ch, Vh, nb, oh, stream, true);
}

int vloc_apply_host_async(vloc_plan p, const void* ch, const void* Vh, int64_t nb, void* oh, void* stream) {
    return apply_host_impl(p, ch, Vh, nb, oh, stream, false);
}

int vloc_device_status(vloc_plan p) {
    if (!p) return VLOC_ERR_ARG;
    if (p->flags & VLOC_HOST_ONLY) return VLOC_OK;
    int h = 0;
    cudaError_t e = cudaMemcpy(&h, p->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e) return cuda_fail(e, "read error flag");
    if (!h) return VLOC_OK;
    if ((e = cudaMemset(p->d_err, 0, sizeof(int)))) return cuda_fail(e, "clear error flag");
    return VLOC_ERR_TIMEOUT;
}

int vloc_profile(vloc_plan p, int enable) {
    if (!p) return VLOC_ERR_ARG;
    if (p->flags & VLOC_HOST_ONLY) return VLOC_ERR_STATE;
    p->prof_on = enable != 0;
    p->prof_recs.clear();
    return VLOC_OK;
}

int vloc_get_profile(vloc_plan p, vloc_kernel_stat* stats) {
    if (!p || !stats) return VLOC_ERR_ARG;
    for (int k = 0; k < VLOC_NKERNELS; ++k) { stats[k].launches = 0; stats[k].total_ms = 0.0; }
    for (const auto& r : p->prof_recs) {
        cudaError_t e = cudaEventSynchronize(p->prof_pool[r.second + 1]);
        if (e) return cuda_fail(e, "profile sync");
        float ms = 0.f;
        if ((e = cudaEventElapsedTime(&ms, p->prof_pool[r.second], p->prof_pool[r.second + 1]))) return cuda_fail(e, "elapsed");
        stats[r.first].launches += 1;
        stats[r.first].total_ms += ms;
    }
    p->prof_recs.clear();
    return VLOC_OK;
}

int vloc_get_launch_count(vloc_plan p, int64_t* count) {
    if (!p || !count) return VLOC_ERR_ARG;
    *count = p->launches;
    return VLOC_OK;
}

int vloc_get_index_map(vloc_plan p, int64_t* gi) {
    if (!p || !gi) return VLOC_ERR_ARG;
    std::memcpy(gi, p->grid_index.data(), (size_t)p->npw_user * sizeof(int64_t));
    return VLOC_OK;
}

int vloc_get_partition(vloc_plan p, int32_t* sp, int32_t* np) {
    if (!p) return VLOC_ERR_ARG;
    if (sp) std::memcpy(sp, p->stick_part.data(), p->stick_part.size() * sizeof(int32_t));
    if (np) *np = p->P;
    return VLOC_OK;
}

int vloc_get_info(vloc_plan p, vloc_info* info) {
    if (!p || !info) return VLOC_ERR_ARG;
    std::memset(info, 0, sizeof(*info));
    info->n1 = p->n1; info->n2 = p->n2; info->n3 = p->n3;
    info->precision = p->dbl ? VLOC_F64 : VLOC_F32;
    info->npw = p->npw_user;
    info->nsticks = p->S; info->nplanes = p->NP; info->nparts = p->P;
    info->lines_per_tile = kLinesPerTile;
    info->path = (p->fast ? 1 : 0) | (p->gamma ? 4 : 0) | (p->df ? 8 : 0) | (p->k3tma_on ? 16 : 0) |
                 (p->lay.xq ? 32 : 0) | (p->lay.zq ? 64 : 0) | (p->gfused ? 128 : 0) |
                 (p->lay.zs && p->fast ? 256 : 0) | (p->lay.runs == 1 && p->fast ? 512 : 0);
    info->chunk_bands = p->chunk;
    info->workspace_bytes = (int64_t)p->ws_bytes;
    for (int a = 0; a < 3; ++a) {
        info->nstages[a] = p->ax.nst[a];
        for (int i = 0; i < 4; ++i) info->radix[a][i] = p->ax.radix[a][i];
    }
    return VLOC_OK;
}

}  // extern "C"

// The plan's index tables, kept on the host for every plan (host-only ones
// included) and never changed after plan creation, so the block lives
// exactly as long as the plan.
int vloc::plan_host_tables(const vloc_plan_s* p, const int** blob, HostTableLayout* lay) {
    if (!p || !blob || !lay) return VLOC_ERR_ARG;
    *blob = p->host_tables.data();
    *lay = p->lay;
    return VLOC_OK;
}

DevTables vloc::device_tables(const int* base, const HostTableLayout& L, int n1, int n2, int n3, long long npw) {
    DevTables t;
    t.stick_row = base + L.o_row;
    t.tile_ptr = base + L.o_tp;
    t.tile_sticks = base + L.o_ts;
    t.tile_pw_ptr = base + L.o_tpp;
    t.tile_pw = reinterpret_cast<const int2*>(base + L.o_tpw);
    t.plane_ptr = base + L.o_plp;
    t.xrow_plane = base + L.o_xr;
    t.S = L.S; t.T = L.T; t.NP = L.NP;
    t.n1 = n1; t.n2 = n2; t.n3 = n3; t.npw = npw;
    t.xq = L.xq;
    t.zq = L.zq;
    t.gok = L.gok;
    t.zd_rows = L.zd_rows;
    t.zdense = base + L.o_zd;
    t.zs = L.zs;
    t.zsh = base + L.o_zs;
    t.runs = L.runs;
    t.run_tab = reinterpret_cast<const int4*>(base + L.o_rn);
    t.err = nullptr;
    t.npw_half = L.nh;
    t.gamma_h_ptr = base + L.o_ghp;
    t.gamma_h = reinterpret_cast<const int4*>(base + L.o_gh);
    return t;
}
