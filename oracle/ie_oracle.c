/*
 * FP64 CPU oracle for the group-by-group far-zone solver.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this file; only the tests, the package smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header or constant generator with the
 * CUDA library.
 *
 * Everything here is the plain definition written out, in double precision,
 * one site pair at a time:
 *
 *   dyadic Green's function D(R)          eq. 5 and eq. 6 (§2.1)
 *   uniform dipole lattice per box         §2.1 ("uniform separation")
 *   field at a site from every dipole      eq. 12 summed as in eq. 14 (§2.2)
 *   translation matrix of one displacement eq. 13 (§2.2)
 *   plane-wave excitation                  §5 (unit amplitude plane wave)
 *
 * Complex numbers cross the interface as interleaved (re, im) doubles.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * eq. 5 and eq. 6:
 *   D(R) = psi(R) { I (1 - j/(kR) - 1/(kR)^2) - Rhat Rhat (1 - 3j/(kR) - 3/(kR)^2) }
 *   psi(R) = -j k eta exp(-j k R) / (4 pi R),   R = r - r'
 * out[2*(3*i+j)] + j*out[2*(3*i+j)+1] = D_ij.
 */
void or_dyad(double k, double eta, const double R[3], double out[18]) {
    double r = sqrt(R[0] * R[0] + R[1] * R[1] + R[2] * R[2]);
    double kr = k * r;
    /* psi = -j k eta (cos kr - j sin kr) / (4 pi r) = k eta (-sin kr - j cos kr) / (4 pi r) */
    double s = k * eta / (4.0 * OR_PI * r);
    double psi_re = -s * sin(kr);
    double psi_im = -s * cos(kr);
    /* a = 1 - j/kr - 1/kr^2 ; b = 1 - 3j/kr - 3/kr^2 */
    double a_re = 1.0 - 1.0 / (kr * kr), a_im = -1.0 / kr;
    double b_re = 1.0 - 3.0 / (kr * kr), b_im = -3.0 / kr;
    double rh[3] = {R[0] / r, R[1] / r, R[2] / r};
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) {
            double t_re = (i == j ? a_re : 0.0) - rh[i] * rh[j] * b_re;
            double t_im = (i == j ? a_im : 0.0) - rh[i] * rh[j] * b_im;
            out[2 * (3 * i + j)] = psi_re * t_re - psi_im * t_im;
            out[2 * (3 * i + j) + 1] = psi_re * t_im + psi_im * t_re;
        }
    }
}

/* Position of dipole site s of a box: the box centre a*(ijk + 1/2 - G/2) plus the
 * cell-centred lattice offset a*((i + 1/2)/L - 1/2) per axis, s = ix + L iy + L^2 iz. */
static void site_pos(double a, int L, int G, const int32_t ijk[3], int s, double p[3]) {
    int ix = s % L, iy = (s / L) % L, iz = s / (L * L);
    int ii[3] = {ix, iy, iz};
    for (int c = 0; c < 3; ++c)
        p[c] = a * ((double)ijk[c] + 0.5 - 0.5 * (double)G) + a * (((double)ii[c] + 0.5) / (double)L - 0.5);
}

void or_site_positions(double a, int L, int G, int64_t nbox, const int32_t *ijk, double *pos) {
    int ns = L * L * L;
    for (int64_t b = 0; b < nbox; ++b)
        for (int s = 0; s < ns; ++s) site_pos(a, L, G, ijk + 3 * b, s, pos + 3 * (b * ns + s));
}

static int cheb(const int32_t *p, const int32_t *q) {
    int m = 0;
    for (int c = 0; c < 3; ++c) {
        int d = abs(p[c] - q[c]);
        if (d > m) m = d;
    }
    return m;
}

/*
 * Brute-force dipole field (eq. 12 summed as in eq. 14), site pair by site pair:
 *   y[t][3l+alpha] = sum over source boxes b, sites q (R != 0) of
 *                    sum_beta D_{alpha beta}(r_l - r_q) x[b][3q+beta]
 * restricted by the box criterion `mode`:
 *   1 = far  (Chebyshev box distance >= 2: the one-box-buffer far zone, Alg. 2)
 *   2 = near (Chebyshev distance <= 1; with self_box_mode = 1 the box itself is skipped)
 *   3 = far + near
 * Only target boxes listed in `targets` (ntarget of them, slots into ijk) are computed.
 * x: [nbox][3 L^3] complex; y: [ntarget][3 L^3] complex (overwritten).
 */
void or_dipole_field(double k, double eta, double a, int L, int G, int64_t nbox, const int32_t *ijk,
                     const double *x, int mode, int self_box_mode, int64_t ntarget,
                     const int64_t *targets, double *y) {
    int ns = L * L * L;
    int nu = 3 * ns;
    double *pos = (double *)malloc(sizeof(double) * 3 * (size_t)nbox * ns);
    or_site_positions(a, L, G, nbox, ijk, pos);
    int64_t nwork = ntarget * ns;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t w = 0; w < nwork; ++w) {
        int64_t ti = w / ns;
        int l = (int)(w % ns);
        int64_t tb = targets[ti];
        const double *rl = pos + 3 * (tb * ns + l);
        double acc[6] = {0, 0, 0, 0, 0, 0};
        double D[18];
        for (int64_t sb = 0; sb < nbox; ++sb) {
            int c = cheb(ijk + 3 * tb, ijk + 3 * sb);
            int use;
            if (c >= 2) use = (mode & 1);
            else use = (mode & 2) && !(self_box_mode == 1 && c == 0);
            if (!use) continue;
            for (int q = 0; q < ns; ++q) {
                if (sb == tb && q == l) continue;   /* coincident dipoles: R = 0 excluded */
                const double *rq = pos + 3 * (sb * ns + q);
                double R[3] = {rl[0] - rq[0], rl[1] - rq[1], rl[2] - rq[2]};
                or_dyad(k, eta, R, D);
                const double *xq = x + 2 * (sb * nu + 3 * q);
                for (int al = 0; al < 3; ++al)
                    for (int be = 0; be < 3; ++be) {
                        double dr = D[2 * (3 * al + be)], di = D[2 * (3 * al + be) + 1];
                        double xr = xq[2 * be], xi = xq[2 * be + 1];
                        acc[2 * al] += dr * xr - di * xi;
                        acc[2 * al + 1] += dr * xi + di * xr;
                    }
            }
        }
        double *yl = y + 2 * (ti * nu + 3 * l);
        for (int i = 0; i < 6; ++i) yl[i] = acc[i];
    }
    free(pos);
}

/*
 * Translation matrix of one box displacement d (eq. 13): the field at the test-box
 * dipole sites l due to unit dipoles at the basis-box sites k, test box = basis box + d,
 *   C[3l+alpha][3k+beta] = D_{alpha beta}(a d + s_l - s_k),
 * with s the lattice offsets.  For d = 0 the coincident entries (l = k) are zero.
 * C: [3L^3][3L^3] complex, row-major.
 */
void or_coupling_block(double k, double eta, double a, int L, const int32_t d[3], double *C) {
    int ns = L * L * L;
    int nu = 3 * ns;
    int32_t zero[3] = {0, 0, 0};
    double D[18];
    for (int l = 0; l < ns; ++l) {
        double pl[3];
        site_pos(a, L, 0, d, l, pl);
        for (int q = 0; q < ns; ++q) {
            double pq[3];
            site_pos(a, L, 0, zero, q, pq);
            double R[3] = {pl[0] - pq[0], pl[1] - pq[1], pl[2] - pq[2]};
            int coincident = (d[0] == 0 && d[1] == 0 && d[2] == 0 && l == q);
            if (!coincident) or_dyad(k, eta, R, D);
            for (int al = 0; al < 3; ++al)
                for (int be = 0; be < 3; ++be) {
                    size_t o = 2 * ((size_t)(3 * l + al) * nu + (3 * q + be));
                    C[o] = coincident ? 0.0 : D[2 * (3 * al + be)];
                    C[o + 1] = coincident ? 0.0 : D[2 * (3 * al + be) + 1];
                }
        }
    }
}

/* Many blocks at once (OpenMP over displacements): C: [nd][3L^3][3L^3] complex. */
void or_coupling_blocks(double k, double eta, double a, int L, int64_t nd, const int32_t *d, double *C) {
    int nu = 3 * L * L * L;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < nd; ++i) or_coupling_block(k, eta, a, L, d + 3 * i, C + 2 * (size_t)i * nu * nu);
}

/*
 * Plane-wave samples at the dipole sites (§5: unit-amplitude uniform plane wave):
 *   e[r][b][3q+alpha] = pol_r[alpha] exp(-j k khat_r . r_q)
 * (exp(+j omega t) convention, so a wave travelling along khat is exp(-j k khat.r)).
 */
void or_plane_wave(double k, double a, int L, int G, int64_t nbox, const int32_t *ijk, int64_t nrhs,
                   const double *khat, const double *pol, double *e) {
    int ns = L * L * L;
    int nu = 3 * ns;
    for (int64_t r = 0; r < nrhs; ++r)
        for (int64_t b = 0; b < nbox; ++b)
            for (int q = 0; q < ns; ++q) {
                double p[3];
                site_pos(a, L, G, ijk + 3 * b, q, p);
                double ph = -k * (khat[3 * r] * p[0] + khat[3 * r + 1] * p[1] + khat[3 * r + 2] * p[2]);
                double cr = cos(ph), ci = sin(ph);
                for (int al = 0; al < 3; ++al) {
                    size_t o = 2 * (((size_t)r * nbox + b) * nu + 3 * q + al);
                    e[o] = pol[3 * r + al] * cr;
                    e[o + 1] = pol[3 * r + al] * ci;
                }
            }
}

/*
 * Far-zone interactions of point-dipole subdomain basis functions by brute force: the
 * original system that the mapping of §2.1 replaces (eq. 3-4 with point sources,
 * tested on the basis functions themselves).  Function f (box fun_box[f]) owns dipoles
 * fun_off[f] .. fun_off[f+1]-1 at absolute positions pos and complex moments mom.
 *   out[f] = sum over dipoles d of f of  mom_d . sum over dipoles e of functions g whose
 *            box is at Chebyshev distance >= 2 from f's box of  D(r_d - r_e) (c_g mom_e)
 * c, out: [n_fun] complex.  want (n_fun flags, or NULL for all): only the flagged outputs
 * are computed, the others are set to 0.
 */
void or_point_dipole_far(double k, double eta, int64_t n_fun, const int64_t *fun_off, const int32_t *fun_box,
                         const int32_t *ijk, const double *pos, const double *mom, const double *c,
                         const uint8_t *want, double *out) {
    int64_t nd = fun_off[n_fun];
    double *w = (double *)malloc(sizeof(double) * 6 * (size_t)(nd > 0 ? nd : 1));
    int32_t *dbox = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nd > 0 ? nd : 1));
    for (int64_t g = 0; g < n_fun; ++g)
        for (int64_t e = fun_off[g]; e < fun_off[g + 1]; ++e) {
            dbox[e] = fun_box[g];
            for (int b = 0; b < 3; ++b) {
                double mr = mom[6 * e + 2 * b], mi = mom[6 * e + 2 * b + 1];
                w[6 * e + 2 * b] = c[2 * g] * mr - c[2 * g + 1] * mi;
                w[6 * e + 2 * b + 1] = c[2 * g] * mi + c[2 * g + 1] * mr;
            }
        }
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t f = 0; f < n_fun; ++f) {
        const int32_t *tf = ijk + 3 * fun_box[f];
        double acc_r = 0.0, acc_i = 0.0;
        if (want && !want[f]) {
            out[2 * f] = 0.0;
            out[2 * f + 1] = 0.0;
            continue;
        }
        for (int64_t d = fun_off[f]; d < fun_off[f + 1]; ++d) {
            double E[6] = {0, 0, 0, 0, 0, 0};
            for (int64_t e = 0; e < nd; ++e) {
                const int32_t *sb = ijk + 3 * dbox[e];
                int cheb = 0;
                for (int q = 0; q < 3; ++q) {
                    int dd = abs(tf[q] - sb[q]);
                    if (dd > cheb) cheb = dd;
                }
                if (cheb < 2) continue;
                double R[3] = {pos[3 * d] - pos[3 * e], pos[3 * d + 1] - pos[3 * e + 1], pos[3 * d + 2] - pos[3 * e + 2]};
                double D[18];
                or_dyad(k, eta, R, D);
                for (int al = 0; al < 3; ++al)
                    for (int be = 0; be < 3; ++be) {
                        double dr = D[2 * (3 * al + be)], di = D[2 * (3 * al + be) + 1];
                        double xr = w[6 * e + 2 * be], xi = w[6 * e + 2 * be + 1];
                        E[2 * al] += dr * xr - di * xi;
                        E[2 * al + 1] += dr * xi + di * xr;
                    }
            }
            for (int al = 0; al < 3; ++al) {
                double mr = mom[6 * d + 2 * al], mi = mom[6 * d + 2 * al + 1];
                acc_r += mr * E[2 * al] - mi * E[2 * al + 1];
                acc_i += mr * E[2 * al + 1] + mi * E[2 * al];
            }
        }
        out[2 * f] = acc_r;
        out[2 * f + 1] = acc_i;
    }
    free(w);
    free(dbox);
}

/* Field of point dipoles at observation points (eq. 4 with point sources):
 * out[o] = sum_s D(obs_o - src_s) mom_s.  obs: [n_obs][3], src: [n_src][3],
 * mom: [n_src][3] complex, out: [n_obs][3] complex (overwritten). */
void or_point_fields(double k, double eta, int64_t n_obs, const double *obs, int64_t n_src, const double *src,
                     const double *mom, double *out) {
#pragma omp parallel for schedule(static)
    for (int64_t o = 0; o < n_obs; ++o) {
        double E[6] = {0, 0, 0, 0, 0, 0};
        for (int64_t s = 0; s < n_src; ++s) {
            double R[3] = {obs[3 * o] - src[3 * s], obs[3 * o + 1] - src[3 * s + 1], obs[3 * o + 2] - src[3 * s + 2]};
            double D[18];
            or_dyad(k, eta, R, D);
            for (int al = 0; al < 3; ++al)
                for (int be = 0; be < 3; ++be) {
                    double dr = D[2 * (3 * al + be)], di = D[2 * (3 * al + be) + 1];
                    double xr = mom[6 * s + 2 * be], xi = mom[6 * s + 2 * be + 1];
                    E[2 * al] += dr * xr - di * xi;
                    E[2 * al + 1] += dr * xi + di * xr;
                }
        }
        for (int i = 0; i < 6; ++i) out[6 * o + i] = E[i];
    }
}
