// internal.h -- structures shared by the host plan builder (plan.cpp) and the
// CUDA kernels (kernels.cu).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace vloc {


// Device-resident index tables of one plan (all int32, one allocation).
//  Sticks are the occupied (h mod n1, k mod n2) z-columns in ascending
//  id (h mod n1) * n2 + (k mod n2) order ("canonical"); plane waves are
//  sorted by (stick, l).  Planes are the occupied h mod n1 values.
struct DevTables {
    const int* stick_pw_ptr;  // [S+1] first canonical plane wave of each stick
    const int* pw_user;       // [npw] caller's index of the q-th canonical plane wave
    const int* pw_z;          // [npw] l mod n3
    const int* stick_row;     // [S]   k mod n2
    const int* part_ptr;      // [P+1] sticks of each part in part_sticks
    const int* part_sticks;   // [S]   canonical stick ids, part by part
    const int* plane_ptr;     // [NP+1] canonical stick range of each plane
    const int* xrow_plane;    // [n1]  plane index of x = h mod n1, or -1
    int S, P, NP;
    int n1, n2, n3;
    long long npw;
};

struct LaunchAxes {
    int n[3];
    int nst[3];
    int radix[3][4];
};

// Kernel kinds (profiling slots).
enum KernelKind { KK_SCATTER_Z = 0, KK_Y_INV = 1, KK_X_V = 2, KK_Y_FWD = 3, KK_Z_GATHER = 4, KK_GRAD_V = 5, KK_AUX = 6 };

// Typed launchers (defined in kernels_impl.cuh, instantiated per precision
// in kernels_f32.cu / kernels_f64.cu).  Every pointer is a device pointer;
// `cyl` is [nb][S][n3], `slab` is [nb][NP][n2][n3], complex of type T.  Each
// launcher returns the cudaError_t of its launch.
template <typename T> struct Launch {
    static size_t smem(int n);
    static size_t smem_grad(int n);
    static int set_limits(int nmax, int optin);
    static int twiddles(void* tw, int n, cudaStream_t st);
    static int k1(const DevTables& t, const LaunchAxes& ax, const void* tw3, const void* coeffs, long long nb,
                  void* cyl, cudaStream_t st);
    static int k2(int sign, const DevTables& t, const LaunchAxes& ax, const void* tw2, long long nb, void* cyl,
                  void* slab, cudaStream_t st);
    static int k3(const DevTables& t, const LaunchAxes& ax, const void* tw1, const void* V, long long nb, void* slab,
                  cudaStream_t st);
    static int k4(const DevTables& t, const LaunchAxes& ax, const void* tw3, const void* cyl, long long nb, void* out,
                  cudaStream_t st);
    static int k3b(const DevTables& t, const LaunchAxes& ax, const void* tw1, const void* sc, const void* sg,
                   long long nb, double* acc, cudaStream_t st);
    static int finish_grad(const double* acc, void* g, long long N, cudaStream_t st);
};
extern template struct Launch<float>;
extern template struct Launch<double>;

// Precision dispatch (kernels.cu): dbl = 0 for float, 1 for double.
int launch_twiddles(int dbl, void* tw, int n, cudaStream_t st);
int launch_k1_scatter_zpass(int dbl, const DevTables& t, const LaunchAxes& ax, const void* tw3, const void* coeffs,
                            long long nb, void* cyl, cudaStream_t st);
int launch_k2_ypass(int dbl, int sign, const DevTables& t, const LaunchAxes& ax, const void* tw2, long long nb,
                    void* cyl, void* slab, cudaStream_t st);
int launch_k3_xpass_v(int dbl, const DevTables& t, const LaunchAxes& ax, const void* tw1, const void* V,
                      long long nb, void* slab, cudaStream_t st);
int launch_k4_zpass_gather(int dbl, const DevTables& t, const LaunchAxes& ax, const void* tw3, const void* cyl,
                           long long nb, void* out, cudaStream_t st);
int launch_k3b_grad_v(int dbl, const DevTables& t, const LaunchAxes& ax, const void* tw1, const void* slab_c,
                      const void* slab_g, long long nb, double* acc, cudaStream_t st);
int launch_finish_grad_v(int dbl, const double* acc, void* gradV, long long N, cudaStream_t st);
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
    size_t o_spp, o_pwu, o_pwz, o_row, o_pp, o_ps, o_plp, o_xr, total;
    int S, P, NP;
};

// Rebuild a plan's index tables from its host-side data (any plan, including
// host-only ones) into `blob` (capacity `cap` ints) without allocating.
// Returns VLOC_OK, or VLOC_ERR_SIZE when `cap` is too small.
int plan_host_tables(const vloc_plan_s* p, int* blob, size_t cap, HostTableLayout* lay);

}  // namespace vloc
