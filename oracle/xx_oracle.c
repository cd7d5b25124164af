/*
 * xx_oracle.c -- plain FP64 CPU oracle for the plane-wave Fock exchange operator.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or call
 * this file: only the tests, the package's smoke check and the benchmark's CPU
 * baseline leg use it.  It shares no code with the CUDA library (its own FFT,
 * its own reciprocal lattice, its own kernel evaluation).
 *
 * What it computes (Hutchinson & Widom, "VASP on a GPU", Sec. "Our
 * Implementation", Eq. 2 and the four nested loops described around it):
 *
 *   for k, q (outer loops over k-points) and target band a, occupied band j
 *   (inner loops over bands), on the real-space FFT grid r_p:
 *       rho(r_p)   = conj(u_qj(r_p)) u_ka(r_p)                    codensity
 *       rhohat(G)  = (1/N) sum_p rho(r_p) exp(-i G.r_p)            forward FFT
 *       What(G)    = v(k - q + G) rhohat(G)                        kernel
 *       W(r_p)     = sum_G What(G) exp(+i G.r_p)                   inverse FFT
 *       acc_ka(r_p) += -(w_qj / N_q) u_qj(r_p) W(r_p)              accumulate
 *   then (V_x c)_ka(G) = (sqrt(Omega)/N) sum_p exp(-i G.r_p) acc_ka(r_p) on the
 *   basis sphere of k, and E_x = (s/2)(1/N_k) sum_ka w_ka Re <c_ka|V_x c_ka>.
 *
 * Orbitals: u_kb(r) = Omega^{-1/2} sum_G c_kb(G) exp(i G.r) (cell-periodic part).
 * Interaction kernels (Hartree units): screened (HSE-type, erfc(mu r)/r)
 *   v(g) = 4 pi/|g|^2 (1 - exp(-|g|^2/(4 mu^2))),  v(0) = pi/mu^2;
 * bare Coulomb 4 pi/|g|^2 with the g = 0 term dropped.
 * Spin-paired: s = 2, occupations w are per spin.
 *
 * Parity pins for every function here live in the tests (direct DFT, brute-force
 * real-space convolution, coefficient-space double convolution, Hermiticity,
 * Parseval, plane-wave lattice sums and the Dirac homogeneous-gas limit,
 * invariances, finite differences).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define ORACLE_SPIN_FACTOR 2.0
#define ORACLE_KERNEL_HSE 0
#define ORACLE_KERNEL_COULOMB 1

/* ------------------------------------------------------------------ FFT --- */

static int smallest_factor(int n)
{
    for (int p = 2; p * p <= n; ++p)
        if (n % p == 0) return p;
    return n;
}

/*
 * Textbook recursive decimation-in-time Cooley-Tukey for any n:
 *   out[k] = sum_{t<n} in[t*stride] * tw[(t*k*tw_step) mod ntop]
 * where tw[e] = exp(sign 2 pi i e / ntop).  n = p*m with p the smallest prime
 * factor; the p sub-transforms of length m are combined by a direct length-p
 * DFT with twiddles (a prime length falls back to the direct DFT).
 */
static void fft_rec(const cplx *in, cplx *out, int n, int stride,
                    const cplx *tw, int ntop, int tw_step, cplx *scratch)
{
    if (n == 1) { out[0] = in[0]; return; }
    int p = smallest_factor(n);
    int m = n / p;
    for (int r = 0; r < p; ++r)
        fft_rec(in + (long)r * stride, out + (long)r * m, m, stride * p, tw, ntop,
                tw_step * p, scratch);
    for (int k = 0; k < m; ++k)
        for (int s = 0; s < p; ++s) {
            int kk = k + s * m;
            cplx acc = 0;
            for (int r = 0; r < p; ++r) {
                long e = ((long)r * kk) % n;
                acc += out[r * m + k] * tw[(e * tw_step) % ntop];
            }
            scratch[kk] = acc;
        }
    memcpy(out, scratch, (size_t)n * sizeof(cplx));
}

static void make_twiddles(cplx *tw, int n, int sign)
{
    for (int e = 0; e < n; ++e) {
        double ang = sign * 2.0 * M_PI * (double)e / (double)n;
        tw[e] = cos(ang) + I * sin(ang);
    }
}

/* In-place unnormalised 3D DFT of data[i3][i2][i1] (i1 fastest).
 * sign = -1: forward (exp(-i G.r)), sign = +1: inverse. */
int oracle_fft3d(cplx *data, int n1, int n2, int n3, int sign)
{
    const int n[3] = {n1, n2, n3};
    const long st[3] = {1, n1, (long)n1 * n2};
    for (int ax = 0; ax < 3; ++ax) {
        const int len = n[ax];
        const int o1 = (ax + 1) % 3, o2 = (ax + 2) % 3;
        const long nlines = (long)n[o1] * n[o2];
        cplx *tw = malloc(sizeof(cplx) * len);
        make_twiddles(tw, len, sign);
#pragma omp parallel
        {
            cplx *line = malloc(sizeof(cplx) * len * 3);
            cplx *res = line + len, *scr = line + 2 * len;
#pragma omp for schedule(static)
            for (long l = 0; l < nlines; ++l) {
                long b = (l % n[o1]) * st[o1] + (l / n[o1]) * st[o2];
                for (int t = 0; t < len; ++t) line[t] = data[b + t * st[ax]];
                fft_rec(line, res, len, 1, tw, len, 1, scr);
                for (int t = 0; t < len; ++t) data[b + t * st[ax]] = res[t];
            }
            free(line);
        }
        free(tw);
    }
    return 0;
}

/* -------------------------------------------------------------- geometry --- */

/* Reciprocal rows b_i = 2 pi (a_j x a_k) / (a_1 . (a_2 x a_3)); returns Omega. */
static double reciprocal_rows(const double A[9], double B[9])
{
    const double *a1 = A, *a2 = A + 3, *a3 = A + 6;
    double c23[3] = {a2[1] * a3[2] - a2[2] * a3[1], a2[2] * a3[0] - a2[0] * a3[2],
                     a2[0] * a3[1] - a2[1] * a3[0]};
    double c31[3] = {a3[1] * a1[2] - a3[2] * a1[1], a3[2] * a1[0] - a3[0] * a1[2],
                     a3[0] * a1[1] - a3[1] * a1[0]};
    double c12[3] = {a1[1] * a2[2] - a1[2] * a2[1], a1[2] * a2[0] - a1[0] * a2[2],
                     a1[0] * a2[1] - a1[1] * a2[0]};
    double vol = a1[0] * c23[0] + a1[1] * c23[1] + a1[2] * c23[2];
    for (int i = 0; i < 3; ++i) {
        B[0 + i] = 2.0 * M_PI * c23[i] / vol;
        B[3 + i] = 2.0 * M_PI * c31[i] / vol;
        B[6 + i] = 2.0 * M_PI * c12[i] / vol;
    }
    return fabs(vol);
}

double oracle_cell_volume(const double lattice[9])
{
    double B[9];
    return reciprocal_rows(lattice, B);
}

/* Signed frequency of FFT index i on a length-n axis (index >= n/2 -> i - n). */
static int freq_of(int i, int n) { return (2 * i >= n) ? i - n : i; }

/* |g|^2 for g = (m + d) . B */
static double g2_of(const double B[9], const double md[3])
{
    double g[3] = {0, 0, 0};
    for (int i = 0; i < 3; ++i)
        for (int c = 0; c < 3; ++c) g[c] += md[i] * B[3 * i + c];
    return g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
}

/* Interaction kernel in reciprocal space; which = 0: v(g), which = 1: dv/dmu. */
static double kernel_value(int kernel, double mu, int which, double g2, int is_zero)
{
    if (kernel == ORACLE_KERNEL_HSE) {
        if (which == 0) {
            if (is_zero) return M_PI / (mu * mu);
            return 4.0 * M_PI / g2 * (-expm1(-g2 / (4.0 * mu * mu)));
        }
        return -2.0 * M_PI / (mu * mu * mu) * exp(-g2 / (4.0 * mu * mu));
    }
    if (which != 0 || is_zero) return 0.0;
    return 4.0 * M_PI / g2;
}

/* v(d + G) on the whole FFT grid, G by signed frequency, d = k - q (fractional). */
int oracle_kernel_grid(const double lattice[9], const int grid[3], const double d[3],
                       int kernel, double mu, int which, double *out)
{
    double B[9];
    reciprocal_rows(lattice, B);
    for (int i3 = 0; i3 < grid[2]; ++i3)
        for (int i2 = 0; i2 < grid[1]; ++i2)
            for (int i1 = 0; i1 < grid[0]; ++i1) {
                double md[3] = {freq_of(i1, grid[0]) + d[0], freq_of(i2, grid[1]) + d[1],
                                freq_of(i3, grid[2]) + d[2]};
                int is_zero = (md[0] == 0.0 && md[1] == 0.0 && md[2] == 0.0);
                double g2 = g2_of(B, md);
                out[((long)i3 * grid[1] + i2) * grid[0] + i1] =
                    kernel_value(kernel, mu, which, g2, is_zero);
            }
    return 0;
}

static long grid_index(const int m[3], const int grid[3])
{
    int i[3];
    for (int a = 0; a < 3; ++a) i[a] = ((m[a] % grid[a]) + grid[a]) % grid[a];
    return ((long)i[2] * grid[1] + i[1]) * grid[0] + i[0];
}

/* u(r_p) = Omega^{-1/2} sum_G c(G) exp(i G.r_p) on the grid (scatter + inverse FFT). */
int oracle_sphere_to_grid(const double lattice[9], const int grid[3], int npw,
                          const int *miller, const cplx *c, cplx *u)
{
    long ntot = (long)grid[0] * grid[1] * grid[2];
    double omega = oracle_cell_volume(lattice);
    memset(u, 0, sizeof(cplx) * ntot);
    for (int g = 0; g < npw; ++g) u[grid_index(miller + 3 * g, grid)] += c[g];
    oracle_fft3d(u, grid[0], grid[1], grid[2], +1);
    double s = 1.0 / sqrt(omega);
    for (long p = 0; p < ntot; ++p) u[p] *= s;
    return 0;
}

/* c(G) = (sqrt(Omega)/N) sum_p exp(-i G.r_p) f(r_p) on the sphere; f is overwritten. */
int oracle_grid_to_sphere(const double lattice[9], const int grid[3], int npw,
                          const int *miller, cplx *f, cplx *c)
{
    long ntot = (long)grid[0] * grid[1] * grid[2];
    double omega = oracle_cell_volume(lattice);
    oracle_fft3d(f, grid[0], grid[1], grid[2], -1);
    double s = sqrt(omega) / (double)ntot;
    for (int g = 0; g < npw; ++g) c[g] = s * f[grid_index(miller + 3 * g, grid)];
    return 0;
}

/* W(r_p) for one pair: W = IFFT(v(d + G) FFT(conj(u_j) u_a) / N). */
int oracle_pair_potential(const double lattice[9], const int grid[3], const double d[3],
                          int kernel, double mu, const cplx *u_j, const cplx *u_a, cplx *W)
{
    long ntot = (long)grid[0] * grid[1] * grid[2];
    double *v = malloc(sizeof(double) * ntot);
    oracle_kernel_grid(lattice, grid, d, kernel, mu, 0, v);
    for (long p = 0; p < ntot; ++p) W[p] = conj(u_j[p]) * u_a[p];
    oracle_fft3d(W, grid[0], grid[1], grid[2], -1);
    for (long p = 0; p < ntot; ++p) W[p] *= v[p] / (double)ntot;
    oracle_fft3d(W, grid[0], grid[1], grid[2], +1);
    free(v);
    return 0;
}

/* ------------------------------------------------------------- operator --- */

/*
 * V_x c for the selected targets.
 *   c_occ [nk][n_occ][npw_max], w_occ [nk][n_occ]; c_tgt [nk][n_tgt][npw_max];
 *   miller [nk][npw_max][3]; kfrac [nk][3]; sel [n_sel][2] = (k, a) pairs, or
 *   NULL for every (k, a) in k-major order; vx_out [n_sel][npw_max] (padding
 *   left zero).  Loop order: k, q (k-points) outside, a, j (bands) inside.
 */
int oracle_apply(const double lattice[9], const int grid[3], int nk, const double *kfrac,
                 const int *npw, int npw_max, const int *miller, int kernel, double mu,
                 const cplx *c_occ, const double *w_occ, int n_occ,
                 const cplx *c_tgt, int n_tgt, const int *sel, int n_sel, cplx *vx_out)
{
    const long ntot = (long)grid[0] * grid[1] * grid[2];
    int *selk = malloc(sizeof(int) * (n_sel > 0 ? n_sel : nk * n_tgt));
    int *sela = malloc(sizeof(int) * (n_sel > 0 ? n_sel : nk * n_tgt));
    if (!sel) {
        n_sel = nk * n_tgt;
        for (int t = 0; t < n_sel; ++t) { selk[t] = t / n_tgt; sela[t] = t % n_tgt; }
    } else {
        for (int t = 0; t < n_sel; ++t) { selk[t] = sel[2 * t]; sela[t] = sel[2 * t + 1]; }
    }
    memset(vx_out, 0, sizeof(cplx) * (size_t)n_sel * npw_max);

    cplx *u_occ = malloc(sizeof(cplx) * ntot * (size_t)n_occ);
    cplx *u_a = malloc(sizeof(cplx) * ntot * (size_t)n_sel);
    cplx *acc = malloc(sizeof(cplx) * ntot * (size_t)n_sel);
    cplx *rho = malloc(sizeof(cplx) * ntot);
    double *v = malloc(sizeof(double) * ntot);

    for (int k = 0; k < nk; ++k) {
        int any = 0;
        for (int t = 0; t < n_sel; ++t) any |= (selk[t] == k);
        if (!any) continue;
        for (int t = 0; t < n_sel; ++t) {
            if (selk[t] != k) continue;
            oracle_sphere_to_grid(lattice, grid, npw[k], miller + (long)k * npw_max * 3,
                                  c_tgt + ((long)k * n_tgt + sela[t]) * npw_max, u_a + ntot * t);
            memset(acc + ntot * t, 0, sizeof(cplx) * ntot);
        }
        for (int q = 0; q < nk; ++q) {
            for (int j = 0; j < n_occ; ++j)
                oracle_sphere_to_grid(lattice, grid, npw[q], miller + (long)q * npw_max * 3,
                                      c_occ + ((long)q * n_occ + j) * npw_max, u_occ + ntot * j);
            double d[3] = {kfrac[3 * k] - kfrac[3 * q], kfrac[3 * k + 1] - kfrac[3 * q + 1],
                           kfrac[3 * k + 2] - kfrac[3 * q + 2]};
            oracle_kernel_grid(lattice, grid, d, kernel, mu, 0, v);
            for (int t = 0; t < n_sel; ++t) {
                if (selk[t] != k) continue;
                const cplx *ua = u_a + ntot * t;
                cplx *acct = acc + ntot * t;
                for (int j = 0; j < n_occ; ++j) {
                    const double wq = w_occ[(long)q * n_occ + j];
                    const cplx *uj = u_occ + ntot * j;
#pragma omp parallel for schedule(static)
                    for (long p = 0; p < ntot; ++p) rho[p] = conj(uj[p]) * ua[p];
                    oracle_fft3d(rho, grid[0], grid[1], grid[2], -1);
#pragma omp parallel for schedule(static)
                    for (long p = 0; p < ntot; ++p) rho[p] *= v[p] / (double)ntot;
                    oracle_fft3d(rho, grid[0], grid[1], grid[2], +1);
                    const double f = -wq / (double)nk;
#pragma omp parallel for schedule(static)
                    for (long p = 0; p < ntot; ++p) acct[p] += f * uj[p] * rho[p];
                }
            }
        }
        for (int t = 0; t < n_sel; ++t)
            if (selk[t] == k)
                oracle_grid_to_sphere(lattice, grid, npw[k], miller + (long)k * npw_max * 3,
                                      acc + ntot * t, vx_out + (long)t * npw_max);
    }
    free(u_occ); free(u_a); free(acc); free(rho); free(v); free(selk); free(sela);
    return 0;
}

/* E_x = (s/2)(1/N_k) sum_{k,a} w_ka <c_ka|V_x c_ka>; returns Re, writes Im to *im_out. */
double oracle_energy_from_vx(int nk, const int *npw, int npw_max, const cplx *c_tgt,
                             const double *w_tgt, int n_tgt, const cplx *vx, double *im_out)
{
    cplx e = 0;
    for (int k = 0; k < nk; ++k)
        for (int a = 0; a < n_tgt; ++a) {
            cplx dot = 0;
            const cplx *c = c_tgt + ((long)k * n_tgt + a) * npw_max;
            const cplx *y = vx + ((long)k * n_tgt + a) * npw_max;
            for (int g = 0; g < npw[k]; ++g) dot += conj(c[g]) * y[g];
            e += w_tgt[(long)k * n_tgt + a] * dot;
        }
    e *= 0.5 * ORACLE_SPIN_FACTOR / (double)nk;
    if (im_out) *im_out = cimag(e);
    return creal(e);
}

/*
 * Pair-sum form (Parseval side of Eq. 2):
 *   S = -(s/2) (Omega / (N_k N_q)) sum_{k,a,q,j} w_ka w_qj sum_G K(k - q + G) |rhohat(G)|^2
 * with K = v (which = 0, equals E_x) or K = dv/dmu (which = 1, equals dE_x/dmu).
 */
double oracle_pair_sum(const double lattice[9], const int grid[3], int nk, const double *kfrac,
                       const int *npw, int npw_max, const int *miller, int kernel, double mu,
                       int which, const cplx *c_occ, const double *w_occ, int n_occ,
                       const cplx *c_tgt, const double *w_tgt, int n_tgt)
{
    const long ntot = (long)grid[0] * grid[1] * grid[2];
    const double omega = oracle_cell_volume(lattice);
    cplx *u_a = malloc(sizeof(cplx) * ntot);
    cplx *u_j = malloc(sizeof(cplx) * ntot);
    cplx *rho = malloc(sizeof(cplx) * ntot);
    double *v = malloc(sizeof(double) * ntot);
    double total = 0.0;
    for (int k = 0; k < nk; ++k)
        for (int q = 0; q < nk; ++q) {
            double d[3] = {kfrac[3 * k] - kfrac[3 * q], kfrac[3 * k + 1] - kfrac[3 * q + 1],
                           kfrac[3 * k + 2] - kfrac[3 * q + 2]};
            oracle_kernel_grid(lattice, grid, d, kernel, mu, which, v);
            for (int a = 0; a < n_tgt; ++a) {
                const double wa = w_tgt[(long)k * n_tgt + a];
                if (wa == 0.0) continue;
                oracle_sphere_to_grid(lattice, grid, npw[k], miller + (long)k * npw_max * 3,
                                      c_tgt + ((long)k * n_tgt + a) * npw_max, u_a);
                for (int j = 0; j < n_occ; ++j) {
                    const double wj = w_occ[(long)q * n_occ + j];
                    if (wj == 0.0) continue;
                    oracle_sphere_to_grid(lattice, grid, npw[q], miller + (long)q * npw_max * 3,
                                          c_occ + ((long)q * n_occ + j) * npw_max, u_j);
                    for (long p = 0; p < ntot; ++p) rho[p] = conj(u_j[p]) * u_a[p];
                    oracle_fft3d(rho, grid[0], grid[1], grid[2], -1);
                    double s = 0.0;
                    for (long p = 0; p < ntot; ++p) {
                        cplx r = rho[p] / (double)ntot;
                        s += v[p] * (creal(r) * creal(r) + cimag(r) * cimag(r));
                    }
                    total += wa * wj * s;
                }
            }
        }
    free(u_a); free(u_j); free(rho); free(v);
    return -0.5 * ORACLE_SPIN_FACTOR * omega / ((double)nk * (double)nk) * total;
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
