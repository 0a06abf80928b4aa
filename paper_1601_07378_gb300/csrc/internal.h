// internal.h -- structures shared by the host plan builder (plan.cpp) and the
// CUDA kernels (kernels.cu).  Not part of the public ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace vloc {


// Device-resident index tables of one plan (int32, one allocation).
//  Sticks are the occupied (h mod n1, k mod n2) z-columns in ascending
//  id (h mod n1) * n2 + (k mod n2) order ("canonical"); planes are the
//  occupied h mod n1 values.  A tile is a run of at most 32 sticks of one
//  partition part (one z-pass CTA); its plane waves form a flat list of
//  {caller index, z | line << 16} entries, sticks in tile order, l ascending.
struct DevTables {
    const int* stick_row;     // [S]   k mod n2
    const int* tile_ptr;      // [T+1] sticks of each tile in tile_sticks
    const int* tile_sticks;   // [S]   canonical stick ids, tile by tile
    const int* tile_pw_ptr;   // [T+1] plane-wave entries of each tile
    const int2* tile_pw;      // [npw] {caller index, z | line << 16}
    const int* plane_ptr;     // [NP+1] canonical stick range of each plane
    const int* xrow_plane;    // [n1]  plane index of x = h mod n1, or -1
    int S, T, NP;
    int n1, n2, n3;
    long long npw;
    // 1 when the occupied x-planes are exactly x = 0..n1/4 and n1 - n1/4 ..
    // n1 - 1 in ascending order (a sphere of radius n1/4 in grid units, the
    // cuboid of Fig. 5 for R = n/4): the x-pass kernels then take the plane
    // of each row at compile time
    int xq;
    // 1 when every plane wave has l mod n3 in 0..n3/4 or n3 - n3/4 .. n3 - 1
    // (|l| <= n3/4): the z-pass kernels then skip the rows outside that band
    int zq;
    // Gamma-point plans whose every G shares a z-pass tile with its -G (gok):
    // per tile [gamma_h_ptr[t], gamma_h_ptr[t+1]) of gamma_h = {h, position
    // of G, position of -G, 0} for the half-list plane waves h whose G lies
    // in the tile (position = z | line << 16; the two coincide at G = 0)
    // dense z-band table of plain plans (zd_rows > 0): [T][zd_rows][32] caller
    // index of the plane wave at each (row, line) of a tile's first-stage row
    // groups that meet the band |l| <= n3/4, or -1
    int zd_rows;
    const int* zdense;
    // class table of plain plans with n3 = 32 C, C <= 4 (zs = 1): [S][n3],
    // entry [s][32 j + m] the caller index of the plane wave of stick s at
    // z = C m + j, or -1 (the warp-register z-passes of kernels_zs.cuh)
    int zs;
    const int* zsh;
    // stick runs of plain FP32 quarter-band plans whose every stick's plane
    // waves are consecutive in the caller's list, l ascending: per tile line
    // [T][32] {caller index of the first, its l, count, 0}; runs = 2: K1
    // addresses its inputs from them, 1: K1 stages them by bulk copies
    // (VLOC_Z_BULK), 0: no runs (K1 reads through the dense table)
    int runs;
    const int4* run_tab;
    int* err;  // the plan's device error flag (set by a bounded wait that ran out), or null
    int gok;
    long long npw_half;  // half-list plane waves per real band (Gamma plans)
    const int* gamma_h_ptr;
    const int4* gamma_h;
};

struct LaunchAxes {
    int n[3];
    int nst[3];
    int radix[3][4];
};

// Tensor map over a plan's slab workspace [ws_bands][NP][n2][2 n3] FP32, box
// {64, 1, NP, 1} (one 32-z tile of every occupied plane at one y), for the
// x-pass kernel's TMA loads and stores; err is the plan's device error flag.
struct K3Tma {
    CUtensorMap map;
    const void* base;   // slab workspace start (band 0 of the map)
    size_t band_bytes;  // NP * n2 * n3 * 8
    int* err;
    int skip_first;     // test aid: block 0 never loads its first tile (its wait runs out)
};

// Kernel kinds (profiling slots).
enum KernelKind { KK_SCATTER_Z = 0, KK_Y_INV = 1, KK_X_V = 2, KK_Y_FWD = 3, KK_Z_GATHER = 4, KK_GRAD_V = 5, KK_AUX = 6, KK_GAMMA = 7, KK_X_TO_GRID = 8,
                  KK_X_FROM_GRID = 9, KK_DENSITY = 10 };

// Typed launchers (defined in kernels_impl.cuh, instantiated per precision
// in kernels_f32.cu / kernels_f64.cu).  Every pointer is a device pointer;
// `cyl` is [nb][S][n3], `slab` is [nb][NP][n2][n3], complex of type T.  Each
// launcher returns the cudaError_t of its launch.
template <typename T> struct Launch {
    static size_t smem(int n);
    static size_t smem_grad(int n);
    static size_t smem_dens(int n);
    static int set_limits(int nmax, int optin);
    static int twiddles(void* tw, int n, cudaStream_t st);
    static int k1(const DevTables& t, const LaunchAxes& ax, const void* tw3, const void* coeffs, long long nb,
                  void* cyl, cudaStream_t st);
    static int k2(int sign, const DevTables& t, const LaunchAxes& ax, const void* tw2, long long nb, void* cyl,
                  void* slab, cudaStream_t st);
    static int k3(const DevTables& t, const LaunchAxes& ax, const void* tw1, const void* V, long long nb, void* slab,
                  cudaStream_t st);
    // out = (1/N) gather + diag * cin (diag, cin: null, or [npw] real and the
    // chunk's coefficients [nb][npw])
    static int k4(const DevTables& t, const LaunchAxes& ax, const void* tw3, const void* cyl, long long nb, void* out,
                  const void* diag, const void* cin, cudaStream_t st);
    static int k3b(const DevTables& t, const LaunchAxes& ax, const void* tw1, const void* sc, const void* sg,
                   long long nb, int ngroups, double* partial, cudaStream_t st);
    static int finish_grad(const double* acc, void* g, long long N, cudaStream_t st);
    // x-pass between the slab and a full grid [nb][n1][n2][n3]: sign +1
    // slab -> grid (inverse), -1 grid -> slab (forward)
    static int k3g(int sign, const DevTables& t, const LaunchAxes& ax, const void* tw1, long long nb, void* slab,
                   void* grid, cudaStream_t st);
    // density x-pass over nb slab bands in groups of bpg (see launch_k3d_density)
    static int k3d(const DevTables& t, const LaunchAxes& ax, const void* tw1, const void* slab, long long nb, int bpg,
                   const void* occ, long long b_base, int pair, long long nreal, double* partial, cudaStream_t st);
};
extern template struct Launch<float>;
extern template struct Launch<double>;

// Compile-time-length launchers (kernels_ct.cuh), instantiated for the axis
// lengths of VLOC_CT_SIZES in kernels_ct_*.cu (FP32).
#define VLOC_CT_SIZES(X) X(24) X(32) X(48) X(60) X(64) X(72) X(80) X(96) X(100) X(120) X(128) X(144)
template <typename T, int N> struct LaunchCT {
    static int k1(const DevTables& t, const void* tw3, const void* coeffs, long long nb, void* cyl, cudaStream_t st);
    static int k2(int sign, const DevTables& t, const void* tw2, long long nb, void* cyl, void* slab, cudaStream_t st);
    // tma: the plan's slab tensor map for the persistent TMA form, or null
    static int k3(const DevTables& t, const void* tw1, const void* V, long long nb, void* slab, const K3Tma* tma,
                  cudaStream_t st);
    static int k4(const DevTables& t, const void* tw3, const void* cyl, long long nb, void* out, const void* diag,
                  const void* cin, cudaStream_t st);
    // Gamma-point pairs (needs DevTables::gok): K1 forms pair p from real
    // bands 2p, 2p + 1 of c [nreal][npw_half]; K4 writes both real bands'
    // results (+ diag times the band when diag is set)
    static int k1g(const DevTables& t, const void* tw3, const void* c, long long npairs, long long nreal, void* cyl,
                   cudaStream_t st);
    static int k4g(const DevTables& t, const void* tw3, const void* cyl, long long npairs, long long nreal, void* out,
                   const void* diag, const void* cin, cudaStream_t st);
    static int k3b(const DevTables& t, const void* tw1, const void* sc, const void* sg, long long nb, int bpg,
                   double* partial, cudaStream_t st);
    static int k3g(int sign, const DevTables& t, const void* tw1, long long nb, void* slab, void* grid, cudaStream_t st);
    static int k3d(const DevTables& t, const void* tw1, const void* slab, long long nb, int bpg, const void* occ,
                   long long b_base, int pair, long long nreal, float* partial, cudaStream_t st);
};

// Compile-time-length launchers for FP64 data (kernels_df.cuh), one value
// per lane slot, 16-line tiles, for the lengths of VLOC_CT_SIZES.  P = 0:
// double-float arithmetic (twiddle tables TwDF [n], V as hi + lo pairs [N],
// cylinder and slab of 16-byte double-float values); P = 1: native FP64
// (twiddles and V as the plan's FP64 tables, double2 cylinder and slab, the
// layout the runtime-radix FP64 kernels use).
template <int P, int N> struct LaunchF64 {
    static int k1(const DevTables& t, const void* tw3, const void* coeffs, long long nb, void* cyl, cudaStream_t st);
    static int k2(int sign, const DevTables& t, const void* tw2, long long nb, void* cyl, void* slab, cudaStream_t st);
    static int k3(const DevTables& t, const void* tw1, const void* V, long long nb, void* slab, cudaStream_t st);
    static int k4(const DevTables& t, const void* tw3, const void* cyl, long long nb, void* out, const void* diag,
                  const void* cin, cudaStream_t st);
};
bool has_df(int n);
bool has_ct(int n);
// TwDF table [n] from an FP64 twiddle table; V [N] FP64 -> hi + lo pairs
int launch_twiddles_df(const void* tw64, void* twdf, int n, cudaStream_t st);
int launch_v_to_df(const void* V, void* Vdf, long long N, cudaStream_t st);

// Precision dispatch (kernels.cu): dbl = 0 for float, 1 for double; `fast`
// selects the compile-time-length kernels when one exists for the axis (FP32
// and native FP64), and fast = 2 with dbl = 1 the double-float kernels (every
// axis must have them: the caller checks has_df).
int launch_twiddles(int dbl, void* tw, int n, cudaStream_t st);
int launch_k1_scatter_zpass(int dbl, int fast, const DevTables& t, const LaunchAxes& ax, const void* tw3, const void* coeffs,
                            long long nb, void* cyl, cudaStream_t st);
int launch_k2_ypass(int dbl, int fast, int sign, const DevTables& t, const LaunchAxes& ax, const void* tw2, long long nb,
                    void* cyl, void* slab, cudaStream_t st);
int launch_k3_xpass_v(int dbl, int fast, const DevTables& t, const LaunchAxes& ax, const void* tw1, const void* V,
                      long long nb, void* slab, cudaStream_t st, const K3Tma* tma = nullptr);
int launch_k4_zpass_gather(int dbl, int fast, const DevTables& t, const LaunchAxes& ax, const void* tw3, const void* cyl,
                           long long nb, void* out, const void* diag, const void* cin, cudaStream_t st);
// dL/dV x-pass over nb bands in groups of at most `bpg` bands; each group's
// partial sum goes to partial[group][N]; launch_reduce_partials then adds the
// groups (in order) into acc.  Returns the groups used via *used.
int launch_k3b_grad_v(int dbl, int fast, const DevTables& t, const LaunchAxes& ax, const void* tw1, const void* slab_c,
                      const void* slab_g, long long nb, int bpg, double* partial, int* used, cudaStream_t st);
// x-pass between slab and full grid (sign +1: slab -> grid, -1: grid -> slab).
int launch_k3_grid(int dbl, int fast, int sign, const DevTables& t, const LaunchAxes& ax, const void* tw1,
                   long long nb, void* slab, void* grid, cudaStream_t st);
// Density x-pass: for slab bands b < nb (global index b_base + b) adds the
// weighted |psi|^2 of groups of at most bpg bands into partial[group][N]
// (occ: device weights or null; pair = 1 for Gamma-point pairs of nreal
// real bands).  Returns the groups used via *used.  The partials are FP32
// (float[group][N] over the same bytes) where density_partials_f32 says so,
// FP64 otherwise.
int launch_k3d_density(int dbl, int fast, const DevTables& t, const LaunchAxes& ax, const void* tw1, const void* slab,
                       long long nb, int bpg, const void* occ, long long b_base, int pair, long long nreal,
                       double* partial, int* used, cudaStream_t st);
// 1 when the density x-pass of this plan is a compile-time-length FP32
// kernel, whose group sums are FP32 values and are stored as such.
int density_partials_f32(int dbl, int fast, const DevTables& t);
size_t density_smem_bytes(int dbl, int n);
int launch_reduce_partials(const double* partial, int ngroups, long long N, double* acc, cudaStream_t st);
// The same over FP32 partials: the groups are added in order in FP32 with
// a compensation word (a sum as accurate as one in twice FP32's precision),
// and the pair is added to acc in FP64 (acc taken as
// zero when `first`); with `out` non-null the total goes there, rounded to
// FP32, instead of to acc.
int launch_reduce_partials_f32(const float* partial, int ngroups, long long N, double* acc, int first, float* out,
                               cudaStream_t st);
int launch_finish_grad_v(int dbl, const double* acc, void* gradV, long long N, cudaStream_t st);
// Gamma-point real mode: pack bands (2p, 2p+1) of c [nb][nh] into complex
// band p of C [np][nfull] over the full list (G, then -G at neg[q]), and
// separate the results U [np][nfull] back into out [nb][nh].
int launch_gamma_pack(int dbl, const void* c, long long nb, long long nh, const int* neg, long long nfull, void* C,
                      long long np, cudaStream_t st);
int launch_gamma_unpack(int dbl, const void* U, long long np, long long nfull, const int* neg, long long nh,
                        void* out, long long nb, const void* diag, const void* c, cudaStream_t st);
// Gamma-point pairs formed / separated inside the FP32 compile-time z-passes
// (DevTables::gok; n3 must have compiled kernels): K1 reads real bands
// c [nreal][npw_half] as npairs pairs, K4 writes them back (+ diag * c)
int launch_k1_gamma(const DevTables& t, const void* tw3, const void* c, long long npairs, long long nreal, void* cyl,
                    cudaStream_t st);
int launch_k4_gamma(const DevTables& t, const void* tw3, const void* cyl, long long npairs, long long nreal, void* out,
                    const void* diag, const void* cin, cudaStream_t st);
int launch_zero_f64(double* p, long long n, cudaStream_t st);
size_t smem_bytes_for(int dbl, int n);
size_t grad_smem_bytes(int dbl, int n);
int set_smem_limits(int dbl, int nmax, int optin);

}  // namespace vloc

struct vloc_plan_s;

namespace vloc {

// Layout of a plan's int32 index tables in one contiguous block (offsets in
// ints), as the kernels read them through DevTables.
struct HostTableLayout {
    size_t o_row, o_tp, o_ts, o_tpp, o_tpw, o_plp, o_xr, total;
    int S, T, NP;
    int xq;  // DevTables::xq
    int zq;  // DevTables::zq
    int gok;  // DevTables::gok
    size_t o_ghp, o_gh, o_zd, o_zs, o_rn;
    int zd_rows;
    int zs;  // DevTables::zs
    int runs;  // DevTables::runs
    long long nh;  // DevTables::npw_half
};

// DevTables pointing into a device copy of the table block at `base`.
DevTables device_tables(const int* base, const HostTableLayout& L, int n1, int n2, int n3, long long npw);

// A plan's index tables as kept on the host for any plan (host-only ones
// included): *blob points into the plan and stays valid, unchanged, until
// the plan is destroyed.  No allocation, no copy.
int plan_host_tables(const vloc_plan_s* p, const int** blob, HostTableLayout* lay);

}  // namespace vloc
