/*
 * FP64 CPU oracle for the local-potential action V_loc|psi> -- TEST
 * INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the bench's
 * CPU-baseline leg load this file's library.  It shares no code, header or
 * table with the CUDA path and is deliberately plain and slow.
 *
 * What it computes (Sec. 2, Eqs. 2-3 and the two-FFT recipe that follows
 * them; grid per Sec. 3.1 / Fig. 1):
 *
 *   1. Scatter: Z = 0 on the n1 x n2 x n3 grid; Z[h mod n1, k mod n2, l mod n3]
 *      = c(G) for every G = (h, k, l) of the plane-wave list.
 *   2. psi(j) = sum_m Z(m) exp(+2 pi i sum_a m_a j_a / n_a), evaluated as a
 *      naive O(n) DFT along each axis in turn (the separable form of the
 *      3-D sum), twiddles from cos/sin of 2 pi ((m*j) mod n) / n in double.
 *   3. u(j) = V(j) psi(j).
 *   4. uhat(m) = (1/N) sum_j u(j) exp(-2 pi i sum_a m_a j_a / n_a).
 *   5. out(G) = uhat[h mod n1, k mod n2, l mod n3].
 *
 * The sign of step 2 follows the convention "a single G maps to e^{+iG.r}";
 * Eq. 2 as printed uses e^{-i(k+G).r}, which is the same operator applied to
 * the negated G-list.  The G->r transform is unnormalised, r->G carries 1/N.
 * The grid is the periodic 2G_cut grid, so the result is the discrete
 * periodic product, wrap-around included (Fig. 1).
 *
 * Gradient (autograd convention grad = dL/dRe + i dL/dIm):
 *   dL/dV(j) = (1/N) sum_n Re( conj(g_n(j)) psi_n(j) ),  g_n = F+ S gout_n.
 *
 * Complex arrays are interleaved (re, im) doubles.  Grid index is
 * (i1*n2 + i2)*n3 + i3 (i3 fastest).  Return codes: 0 ok, -2 bad size,
 * -3 bad G-list (index out of range or duplicate), -5 out of memory.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_ERR_SIZE (-2)
#define ORC_ERR_GLIST (-3)
#define ORC_ERR_ALLOC (-5)

static int valid_miller(int h, int n) { return h >= -(n / 2) && h <= (n + 1) / 2 - 1; }
static int64_t pmod(int64_t a, int64_t n) { int64_t r = a % n; return r < 0 ? r + n : r; }

/* Step 1's map G -> grid index (Eqs. 2-3: each plane wave is one grid point). */
int oracle_index_map(int n1, int n2, int n3, const int32_t* g, int64_t npw, int64_t* idx)
{
    if (n1 < 1 || n2 < 1 || n3 < 1) return ORC_ERR_SIZE;
    int64_t N = (int64_t)n1 * n2 * n3;
    unsigned char* seen = (unsigned char*)calloc((size_t)N, 1);
    if (!seen) return ORC_ERR_ALLOC;
    int rc = ORC_OK;
    for (int64_t p = 0; p < npw; ++p) {
        int h = g[3 * p], k = g[3 * p + 1], l = g[3 * p + 2];
        if (!valid_miller(h, n1) || !valid_miller(k, n2) || !valid_miller(l, n3)) { rc = ORC_ERR_GLIST; break; }
        int64_t j = (pmod(h, n1) * n2 + pmod(k, n2)) * n3 + pmod(l, n3);
        if (seen[j]) { rc = ORC_ERR_GLIST; break; }
        seen[j] = 1;
        idx[p] = j;
    }
    free(seen);
    return rc;
}

/* Naive 1-D DFT of every line of the grid along one axis:
 * out[k] = sum_m in[m] exp(sign * 2 pi i m k / n). */
static void dft_axis(double* a, const int n[3], int axis, int sign)
{
    int len = n[axis];
    double* cs = (double*)malloc(sizeof(double) * len);
    double* sn = (double*)malloc(sizeof(double) * len);
    double* tmp = (double*)malloc(sizeof(double) * 2 * len);
    for (int j = 0; j < len; ++j) {
        double ang = 2.0 * M_PI * (double)j / (double)len;
        cs[j] = cos(ang);
        sn[j] = (double)sign * sin(ang);
    }
    int64_t stride = axis == 0 ? (int64_t)n[1] * n[2] : (axis == 1 ? n[2] : 1);
    /* lines: every index with the axis coordinate set to 0 */
    for (int i1 = 0; i1 < (axis == 0 ? 1 : n[0]); ++i1)
        for (int i2 = 0; i2 < (axis == 1 ? 1 : n[1]); ++i2)
            for (int i3 = 0; i3 < (axis == 2 ? 1 : n[2]); ++i3) {
                int64_t base = ((int64_t)i1 * n[1] + i2) * n[2] + i3;
                for (int m = 0; m < len; ++m) {
                    tmp[2 * m] = a[2 * (base + m * stride)];
                    tmp[2 * m + 1] = a[2 * (base + m * stride) + 1];
                }
                for (int k = 0; k < len; ++k) {
                    double re = 0.0, im = 0.0;
                    for (int m = 0; m < len; ++m) {
                        int t = (int)(((int64_t)m * k) % len);
                        re += tmp[2 * m] * cs[t] - tmp[2 * m + 1] * sn[t];
                        im += tmp[2 * m] * sn[t] + tmp[2 * m + 1] * cs[t];
                    }
                    a[2 * (base + k * stride)] = re;
                    a[2 * (base + k * stride) + 1] = im;
                }
            }
    free(cs); free(sn); free(tmp);
}

/* Exposed for the compact-support checks: one naive DFT pass along `axis`
 * (0 = i1, 1 = i2, 2 = i3) of `nb` full grids, in place. */
int oracle_axis_dft(int n1, int n2, int n3, double* grids, int64_t nb, int axis, int sign, int nthreads)
{
    int n[3] = {n1, n2, n3};
    int64_t N = (int64_t)n1 * n2 * n3;
    if (axis < 0 || axis > 2 || (sign != 1 && sign != -1)) return ORC_ERR_SIZE;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t b = 0; b < nb; ++b) dft_axis(grids + 2 * N * b, n, axis, sign);
    return ORC_OK;
}

/* Steps 1-2 for one band: psi = F+ S c on the full grid. */
static void to_real_one(const int n[3], const int64_t* idx, int64_t npw, const double* c, double* psi)
{
    int64_t N = (int64_t)n[0] * n[1] * n[2];
    memset(psi, 0, sizeof(double) * 2 * N);
    for (int64_t p = 0; p < npw; ++p) {
        psi[2 * idx[p]] = c[2 * p];
        psi[2 * idx[p] + 1] = c[2 * p + 1];
    }
    dft_axis(psi, n, 0, +1);
    dft_axis(psi, n, 1, +1);
    dft_axis(psi, n, 2, +1);
}

int oracle_to_real(int n1, int n2, int n3, const int32_t* g, int64_t npw, const double* c,
                   int64_t nb, double* psi, int nthreads)
{
    int n[3] = {n1, n2, n3};
    int64_t N = (int64_t)n1 * n2 * n3;
    int64_t* idx = (int64_t*)malloc(sizeof(int64_t) * (npw > 0 ? npw : 1));
    if (!idx) return ORC_ERR_ALLOC;
    int rc = oracle_index_map(n1, n2, n3, g, npw, idx);
    if (rc) { free(idx); return rc; }
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t b = 0; b < nb; ++b) to_real_one(n, idx, npw, c + 2 * npw * b, psi + 2 * N * b);
    free(idx);
    return ORC_OK;
}

/* Steps 1-5: out = (1/N) S^T F- diag(V) F+ S c, band by band. */
int oracle_apply(int n1, int n2, int n3, const int32_t* g, int64_t npw, const double* c,
                 const double* V, int64_t nb, double* out, int nthreads)
{
    int n[3] = {n1, n2, n3};
    int64_t N = (int64_t)n1 * n2 * n3;
    int64_t* idx = (int64_t*)malloc(sizeof(int64_t) * (npw > 0 ? npw : 1));
    if (!idx) return ORC_ERR_ALLOC;
    int rc = oracle_index_map(n1, n2, n3, g, npw, idx);
    if (rc) { free(idx); return rc; }
    int fail = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t b = 0; b < nb; ++b) {
        double* w = (double*)malloc(sizeof(double) * 2 * N);
        if (!w) { fail = 1; continue; }
        to_real_one(n, idx, npw, c + 2 * npw * b, w);
        for (int64_t j = 0; j < N; ++j) { w[2 * j] *= V[j]; w[2 * j + 1] *= V[j]; }
        dft_axis(w, n, 0, -1);
        dft_axis(w, n, 1, -1);
        dft_axis(w, n, 2, -1);
        double* o = out + 2 * npw * b;
        for (int64_t p = 0; p < npw; ++p) {
            o[2 * p] = w[2 * idx[p]] / (double)N;
            o[2 * p + 1] = w[2 * idx[p] + 1] / (double)N;
        }
        free(w);
    }
    free(idx);
    return fail ? ORC_ERR_ALLOC : ORC_OK;
}

/* dL/dV(j) = (1/N) sum_b Re(conj(g_b(j)) psi_b(j)), g_b = F+ S gout_b,
 * psi_b = F+ S c_b.  dV is overwritten (float64 [N]). */
int oracle_grad_V(int n1, int n2, int n3, const int32_t* g, int64_t npw, const double* c,
                  const double* gout, int64_t nb, double* dV, int nthreads)
{
    int n[3] = {n1, n2, n3};
    int64_t N = (int64_t)n1 * n2 * n3;
    int64_t* idx = (int64_t*)malloc(sizeof(int64_t) * (npw > 0 ? npw : 1));
    if (!idx) return ORC_ERR_ALLOC;
    int rc = oracle_index_map(n1, n2, n3, g, npw, idx);
    if (rc) { free(idx); return rc; }
    double* parts = (double*)calloc((size_t)(N * (nb > 0 ? nb : 1)), sizeof(double));
    if (!parts) { free(idx); return ORC_ERR_ALLOC; }
    int fail = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t b = 0; b < nb; ++b) {
        double* psi = (double*)malloc(sizeof(double) * 2 * N);
        double* gr = (double*)malloc(sizeof(double) * 2 * N);
        if (!psi || !gr) { fail = 1; free(psi); free(gr); continue; }
        to_real_one(n, idx, npw, c + 2 * npw * b, psi);
        to_real_one(n, idx, npw, gout + 2 * npw * b, gr);
        double* pb = parts + N * b;
        for (int64_t j = 0; j < N; ++j)
            pb[j] = (gr[2 * j] * psi[2 * j] + gr[2 * j + 1] * psi[2 * j + 1]) / (double)N;
        free(psi); free(gr);
    }
    /* sum over bands in band order (deterministic) */
    for (int64_t j = 0; j < N; ++j) {
        double s = 0.0;
        for (int64_t b = 0; b < nb; ++b) s += parts[N * b + j];
        dV[j] = s;
    }
    free(parts); free(idx);
    return fail ? ORC_ERR_ALLOC : ORC_OK;
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
