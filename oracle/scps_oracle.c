/*
 * FP64 CPU oracle for ratchet-and-pawl biased Langevin dynamics (rMD).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may call this code:
 * only the test-suite, the package smoke check and the CPU-baseline leg of the
 * benchmark load it. It shares no code, header, table or constant generator
 * with the CUDA library; both receive the same seeded inputs from the `synth`
 * package and compute everything else on their own.
 *
 * Everything is plain double-precision loops in the order the paper states
 * the computation, with no blocking, fusion or reordering:
 *
 *   Langevin equation ........................ Eq. (Lang)
 *   ratchet-and-pawl bias force .............. Eq. (FrMD); theta(0) = 1
 *   collective coordinate z(X) ............... Eq. (zrMD)
 *   contact-map entries C_ij ................. Eq. (Cij)
 *   z_m = running minimum of z, z_m(0)=z(X0) . Sec. "Ratchet-and-Pawl MD and Bias Functional"
 *   bias functional T[X] ..................... Eq. for T in the same section
 *   overdamped Langevin (toy model) .......... Sec. "Diffusion in a 2-dimensional asymmetric funnel"
 *
 * The paper leaves the integrator, the synthetic force field, the noise
 * generator and the cutoff treatment open; the readings taken here are:
 *   - underdamped runs use BAOAB (Leimkuhler & Matthews 2013) in the order
 *     B(dt/2) A(dt/2) O(dt) A(dt/2) [force] B(dt/2);
 *   - overdamped runs use Euler-Maruyama x += (dt/gamma) F + sqrt(2 kT dt/gamma) xi;
 *   - noise: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) keyed by the
 *     64-bit seed, counter (atom, replica, step, stream), turned into normals by
 *     Box-Muller with u1 = (a + 1) 2^-32 in (0, 1] and u2 = b 2^-32;
 *   - pair potential: Lennard-Jones (Lorentz-Berthelot) plus Coulomb
 *     (distance-dependent dielectric eps_r = k_dd r, reaction field, or plain),
 *     shifted-force at the cutoff r_c so energy and force vanish there;
 *   - C_ij uses the exact rewrite (1 - u^3)/(1 - u^5) =
 *     (1 + u + u^2)/(1 + u + u^2 + u^3 + u^4), u = (r/r0)^2, which removes the
 *     0/0 at r = r0 (where C = 3/5);
 *   - a bias step with z >= z_m applies F = -k_R (z - z_m) grad z; with
 *     z < z_m it sets z_m = z and applies no bias.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (SC'11, "Parallel random numbers: as easy as 1, 2, 3")        */
/* ------------------------------------------------------------------------- */
static void philox_round(uint32_t c[4], const uint32_t k[2]) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c[1] ^ k[0];
    const uint32_t n2 = hi0 ^ c[3] ^ k[1];
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
}

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k[0] += 0x9E3779B9u;
            k[1] += 0xBB67AE85u;
        }
        philox_round(c, k);
    }
    memcpy(out, c, sizeof(c));
}

/* Four standard normals for (seed; atom, replica, step, stream). */
void orc_normals4(uint64_t seed, uint32_t atom, uint32_t replica, uint32_t step,
                  uint32_t stream, double out[4]) {
    const uint32_t ctr[4] = {atom, replica, step, stream};
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t r[4];
    orc_philox4x32_10(ctr, key, r);
    for (int p = 0; p < 2; ++p) {
        const double u1 = ((double)r[2 * p] + 1.0) * (1.0 / 4294967296.0);
        const double u2 = (double)r[2 * p + 1] * (1.0 / 4294967296.0);
        const double rad = sqrt(-2.0 * log(u1));
        out[2 * p] = rad * cos(2.0 * ORC_PI * u2);
        out[2 * p + 1] = rad * sin(2.0 * ORC_PI * u2);
    }
}

/* ------------------------------------------------------------------------- */
/* Force field                                                                */
/* ------------------------------------------------------------------------- */
enum { ORC_ELEC_NONE = 0, ORC_ELEC_DDIEL = 1, ORC_ELEC_RF = 2, ORC_ELEC_PLAIN = 3 };

typedef struct {
    int n;
    const double *mass, *charge, *sigma, *eps;
    int nb;
    const int32_t *bonds;      /* nb x 2 */
    const double *b0, *kb;
    int na;
    const int32_t *angles;     /* na x 3, centre in the middle */
    const double *th0, *kth;
    int ne;
    const int32_t *excl;       /* ne x 2, excluded pairs */
    double cutoff;
    int elec;
    double k_dd;               /* distance-dependent dielectric: eps_r = k_dd * r (r in nm) */
    double eps_rf;             /* reaction-field dielectric */
    double coulomb_f;          /* 138.935458 kJ mol^-1 nm e^-2 */
    double box;                /* > 0: cubic periodic box edge, minimum image */
} orc_ff;

/* Energy terms, in this order. */
enum { ORC_E_BOND = 0, ORC_E_ANGLE, ORC_E_LJ, ORC_E_COUL, ORC_E_N };

/* Pair potential phi(r) and its derivative for one pair (before the shift). */
static void pair_phi(const orc_ff* ff, int i, int j, double r, double* lj, double* dlj,
                     double* cl, double* dcl) {
    const double sig = 0.5 * (ff->sigma[i] + ff->sigma[j]);
    const double eps = sqrt(ff->eps[i] * ff->eps[j]);
    const double sr6 = pow(sig / r, 6.0);
    *lj = 4.0 * eps * (sr6 * sr6 - sr6);
    *dlj = -24.0 * eps * (2.0 * sr6 * sr6 - sr6) / r;
    const double qq = ff->coulomb_f * ff->charge[i] * ff->charge[j];
    *cl = 0.0;
    *dcl = 0.0;
    if (ff->elec == ORC_ELEC_DDIEL) {
        *cl = qq / (ff->k_dd * r * r);
        *dcl = -2.0 * qq / (ff->k_dd * r * r * r);
    } else if (ff->elec == ORC_ELEC_RF) {
        const double rc = ff->cutoff;
        const double krf = (ff->eps_rf - 1.0) / ((2.0 * ff->eps_rf + 1.0) * rc * rc * rc);
        const double crf = 1.0 / rc + krf * rc * rc;
        *cl = qq * (1.0 / r + krf * r * r - crf);
        *dcl = qq * (-1.0 / (r * r) + 2.0 * krf * r);
    } else if (ff->elec == ORC_ELEC_PLAIN) {
        *cl = qq / r;
        *dcl = -qq / (r * r);
    }
}

static int is_excluded(const orc_ff* ff, const int32_t* ex_off, const int32_t* ex_idx, int i,
                       int j) {
    for (int k = ex_off[i]; k < ex_off[i + 1]; ++k)
        if (ex_idx[k] == j) return 1;
    return 0;
}

/* CSR of excluded partners per atom (both directions). */
static void build_exclusions(const orc_ff* ff, int32_t** off, int32_t** idx) {
    int32_t* cnt = (int32_t*)calloc((size_t)ff->n + 1, sizeof(int32_t));
    for (int e = 0; e < ff->ne; ++e) {
        cnt[ff->excl[2 * e] + 1]++;
        cnt[ff->excl[2 * e + 1] + 1]++;
    }
    for (int i = 0; i < ff->n; ++i) cnt[i + 1] += cnt[i];
    int32_t* fill = (int32_t*)malloc(sizeof(int32_t) * (size_t)(ff->n + 1));
    memcpy(fill, cnt, sizeof(int32_t) * (size_t)(ff->n + 1));
    int32_t* list = (int32_t*)malloc(sizeof(int32_t) * (size_t)(2 * ff->ne + 1));
    for (int e = 0; e < ff->ne; ++e) {
        const int a = ff->excl[2 * e], b = ff->excl[2 * e + 1];
        list[fill[a]++] = b;
        list[fill[b]++] = a;
    }
    free(fill);
    *off = cnt;
    *idx = list;
}

static void min_image(const orc_ff* ff, double d[3]) {
    if (ff->box > 0.0)
        for (int k = 0; k < 3; ++k) d[k] -= ff->box * nearbyint(d[k] / ff->box);
}

/* One non-bonded pair (i, j), j != i, with separation d = x_j - x_i.
 * Adds energies and forces (shifted-force form, Allen & Tildesley). */
static void add_pair(const orc_ff* ff, int i, int j, const double d[3], double* F, double* E) {
    const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    const double rc = ff->cutoff;
    if (r2 >= rc * rc) return;
    const double r = sqrt(r2);
    double lj, dlj, cl, dcl, ljc, dljc, clc, dclc;
    pair_phi(ff, i, j, r, &lj, &dlj, &cl, &dcl);
    pair_phi(ff, i, j, rc, &ljc, &dljc, &clc, &dclc);
    if (E) {
        E[ORC_E_LJ] += lj - ljc - (r - rc) * dljc;
        E[ORC_E_COUL] += cl - clc - (r - rc) * dclc;
    }
    if (F) {
        /* F_i = phi_sf'(r) d / r, F_j = -F_i */
        const double dphi = (dlj - dljc) + (dcl - dclc);
        for (int k = 0; k < 3; ++k) {
            const double f = dphi * d[k] / r;
            F[3 * i + k] += f;
            F[3 * j + k] -= f;
        }
    }
}

static void bonded_terms(const orc_ff* ff, const double* x, double* F, double* E) {
    for (int b = 0; b < ff->nb; ++b) {
        const int i = ff->bonds[2 * b], j = ff->bonds[2 * b + 1];
        double d[3];
        for (int k = 0; k < 3; ++k) d[k] = x[3 * j + k] - x[3 * i + k];
        min_image(ff, d);
        const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        const double dr = r - ff->b0[b];
        if (E) E[ORC_E_BOND] += 0.5 * ff->kb[b] * dr * dr;
        if (F)
            for (int k = 0; k < 3; ++k) {
                const double f = ff->kb[b] * dr * d[k] / r;
                F[3 * i + k] += f;
                F[3 * j + k] -= f;
            }
    }
    for (int a = 0; a < ff->na; ++a) {
        const int i = ff->angles[3 * a], j = ff->angles[3 * a + 1], l = ff->angles[3 * a + 2];
        double u[3], w[3];
        for (int k = 0; k < 3; ++k) {
            u[k] = x[3 * i + k] - x[3 * j + k];
            w[k] = x[3 * l + k] - x[3 * j + k];
        }
        min_image(ff, u);
        min_image(ff, w);
        const double ru = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        const double rw = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
        const double c[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2],
                             u[0] * w[1] - u[1] * w[0]};
        const double sn = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
        const double cs = u[0] * w[0] + u[1] * w[1] + u[2] * w[2];
        const double th = atan2(sn, cs);
        const double dth = th - ff->th0[a];
        if (E) E[ORC_E_ANGLE] += 0.5 * ff->kth[a] * dth * dth;
        if (F) {
            /* d theta / d x_i = (cos th u_hat - w_hat) / (|u| sin th), same for x_l */
            const double sin_t = sn / (ru * rw), cos_t = cs / (ru * rw);
            const double g = -ff->kth[a] * dth;
            for (int k = 0; k < 3; ++k) {
                const double uh = u[k] / ru, wh = w[k] / rw;
                const double gi = (cos_t * uh - wh) / (ru * sin_t);
                const double gl = (cos_t * wh - uh) / (rw * sin_t);
                F[3 * i + k] += g * gi;
                F[3 * l + k] += g * gl;
                F[3 * j + k] -= g * (gi + gl);
            }
        }
    }
}

/* Brute force: bonded terms plus every non-excluded pair i < j within r_c.
 * F (n x 3, may be NULL) and E (ORC_E_N, may be NULL) are overwritten. */
void orc_forces(const orc_ff* ff, const double* x, double* F, double* E) {
    if (F) memset(F, 0, sizeof(double) * 3 * (size_t)ff->n);
    if (E) memset(E, 0, sizeof(double) * ORC_E_N);
    int32_t *off, *idx;
    build_exclusions(ff, &off, &idx);
    bonded_terms(ff, x, F, E);
    for (int i = 0; i < ff->n; ++i)
        for (int j = i + 1; j < ff->n; ++j) {
            if (is_excluded(ff, off, idx, i, j)) continue;
            double d[3];
            for (int k = 0; k < 3; ++k) d[k] = x[3 * j + k] - x[3 * i + k];
            min_image(ff, d);
            add_pair(ff, i, j, d, F, E);
        }
    free(off);
    free(idx);
}

/* Same result through a cell list (cells of edge >= r_c; periodic box only):
 * every pair i < j whose cells are neighbours is visited once. */
int orc_forces_cells(const orc_ff* ff, const double* x, double* F, double* E) {
    if (ff->box <= 0.0) return -1;
    const int nc = (int)floor(ff->box / ff->cutoff);
    if (nc < 3) {
        orc_forces(ff, x, F, E);
        return 0;
    }
    if (F) memset(F, 0, sizeof(double) * 3 * (size_t)ff->n);
    if (E) memset(E, 0, sizeof(double) * ORC_E_N);
    int32_t *off, *idx;
    build_exclusions(ff, &off, &idx);
    bonded_terms(ff, x, F, E);
    const int ncell = nc * nc * nc;
    int32_t* head = (int32_t*)malloc(sizeof(int32_t) * (size_t)ncell);
    int32_t* next = (int32_t*)malloc(sizeof(int32_t) * (size_t)ff->n);
    int32_t* cell_of = (int32_t*)malloc(sizeof(int32_t) * (size_t)ff->n);
    for (int c = 0; c < ncell; ++c) head[c] = -1;
    for (int i = ff->n - 1; i >= 0; --i) {
        int ci[3];
        for (int k = 0; k < 3; ++k) {
            double s = x[3 * i + k] / ff->box;
            s -= floor(s);
            int q = (int)(s * nc);
            if (q >= nc) q = nc - 1;
            ci[k] = q;
        }
        const int c = (ci[0] * nc + ci[1]) * nc + ci[2];
        cell_of[i] = c;
        next[i] = head[c];
        head[c] = i;
    }
    for (int i = 0; i < ff->n; ++i) {
        const int c = cell_of[i];
        const int cx = c / (nc * nc), cy = (c / nc) % nc, cz = c % nc;
        for (int ox = -1; ox <= 1; ++ox)
            for (int oy = -1; oy <= 1; ++oy)
                for (int oz = -1; oz <= 1; ++oz) {
                    const int qx = (cx + ox + nc) % nc, qy = (cy + oy + nc) % nc,
                              qz = (cz + oz + nc) % nc;
                    for (int j = head[(qx * nc + qy) * nc + qz]; j >= 0; j = next[j]) {
                        if (j <= i || is_excluded(ff, off, idx, i, j)) continue;
                        double d[3];
                        for (int k = 0; k < 3; ++k) d[k] = x[3 * j + k] - x[3 * i + k];
                        min_image(ff, d);
                        add_pair(ff, i, j, d, F, E);
                    }
                }
    }
    free(head);
    free(next);
    free(cell_of);
    free(off);
    free(idx);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Native contacts, z(X) and the ratchet (Eqs. Cij, zrMD, FrMD)                */
/* ------------------------------------------------------------------------- */
/* C(r) of Eq. (Cij) with u = (r/r0)^2, written as (1+u+u^2)/(1+u+u^2+u^3+u^4). */
double orc_contact_C(double r, double r0) {
    const double u = (r / r0) * (r / r0);
    const double num = 1.0 + u + u * u;
    return num / (num + u * u * u + u * u * u * u);
}

/* The raw ratio of Eq. (Cij), for the pin tests only (0/0 at r = r0). */
double orc_contact_C_raw(double r, double r0) {
    const double s = r / r0;
    return (1.0 - pow(s, 6.0)) / (1.0 - pow(s, 10.0));
}

/* dC/du for the rewritten form. */
static double contact_dC_du(double u) {
    const double num = 1.0 + u + u * u;
    const double den = num + u * u * u + u * u * u * u;
    const double dnum = 1.0 + 2.0 * u;
    const double dden = dnum + 3.0 * u * u + 4.0 * u * u * u;
    return (dnum * den - num * dden) / (den * den);
}

typedef struct {
    int nc;
    const int32_t* pairs;  /* nc x 2 */
    const double* C0;      /* nc: native map entries C_ij(X_N) */
    double r0;
    double k_R;
    double box;            /* > 0: minimum image */
} orc_bias;

/* C0_ij = C_ij(X_N) for the listed pairs. */
void orc_native_map(int nc, const int32_t* pairs, double r0, double box, const double* xN,
                    double* C0) {
    for (int p = 0; p < nc; ++p) {
        const int i = pairs[2 * p], j = pairs[2 * p + 1];
        double d[3];
        for (int k = 0; k < 3; ++k) {
            d[k] = xN[3 * j + k] - xN[3 * i + k];
            if (box > 0.0) d[k] -= box * nearbyint(d[k] / box);
        }
        const double u = (d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) / (r0 * r0);
        const double num = 1.0 + u + u * u;
        C0[p] = num / (num + u * u * u + u * u * u * u);
    }
}

/* z(X) = sum over listed pairs of (C_ij(X) - C0_ij)^2, summed in list order;
 * grad (n x 3, may be NULL) is overwritten with grad z. */
double orc_z(const orc_bias* b, int n, const double* x, double* grad) {
    if (grad) memset(grad, 0, sizeof(double) * 3 * (size_t)n);
    double z = 0.0;
    for (int p = 0; p < b->nc; ++p) {
        const int i = b->pairs[2 * p], j = b->pairs[2 * p + 1];
        double d[3];
        for (int k = 0; k < 3; ++k) {
            d[k] = x[3 * j + k] - x[3 * i + k];
            if (b->box > 0.0) d[k] -= b->box * nearbyint(d[k] / b->box);
        }
        const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        const double u = r2 / (b->r0 * b->r0);
        const double num = 1.0 + u + u * u;
        const double C = num / (num + u * u * u + u * u * u * u);
        const double dev = C - b->C0[p];
        z += dev * dev;
        if (grad) {
            /* d/dx_j of (C - C0)^2 = 2 (C - C0) C'(u) 2 d / r0^2; x_i gets the negative */
            const double g = 2.0 * dev * contact_dC_du(u) * 2.0 / (b->r0 * b->r0);
            for (int k = 0; k < 3; ++k) {
                grad[3 * j + k] += g * d[k];
                grad[3 * i + k] -= g * d[k];
            }
        }
    }
    return z;
}

/* Ratchet of Eq. (FrMD): given z at the current configuration and the running
 * minimum *zm, update *zm and return the factor s such that F_bias = s grad z.
 * theta(0) = 1, so z == z_m keeps the (zero-valued) bias branch. */
double orc_ratchet(double z, double* zm, double k_R) {
    if (z < *zm) {
        *zm = z;
        return 0.0;
    }
    return -k_R * (z - *zm);
}

/* ------------------------------------------------------------------------- */
/* Full forces of one replica: physical + bias, with the z_m update            */
/* ------------------------------------------------------------------------- */
typedef struct {
    double z, zm, epot, fbias2_over_m; /* sum_i |F_bias,i|^2 / m_i */
} orc_eval;

static void eval_all(const orc_ff* ff, const orc_bias* b, const double* x, double* F,
                     double* work, double* zm, orc_eval* ev) {
    double E[ORC_E_N];
    orc_forces(ff, x, F, E);
    ev->epot = E[0] + E[1] + E[2] + E[3];
    ev->z = 0.0;
    ev->fbias2_over_m = 0.0;
    if (b && b->nc > 0) {
        const double z = orc_z(b, ff->n, x, work);
        const double s = orc_ratchet(z, zm, b->k_R);
        ev->z = z;
        for (int i = 0; i < ff->n; ++i) {
            double f2 = 0.0;
            for (int k = 0; k < 3; ++k) {
                const double fb = s * work[3 * i + k];
                F[3 * i + k] += fb;
                f2 += fb * fb;
            }
            ev->fbias2_over_m += f2 / ff->mass[i];
        }
    }
    ev->zm = *zm;
}

/* Forces (physical + bias) and energy of one configuration at a given z_m,
 * with the z_m update of the ratchet applied to *zm. */
void orc_eval_replica(const orc_ff* ff, const orc_bias* b, const double* x, double* F,
                      double* zm, double* z_out, double* epot_out) {
    double* work = (double*)malloc(sizeof(double) * 3 * (size_t)ff->n);
    orc_eval ev;
    eval_all(ff, b, x, F, work, zm, &ev);
    if (z_out) *z_out = ev.z;
    if (epot_out) *epot_out = ev.epot;
    free(work);
}

/* ------------------------------------------------------------------------- */
/* BAOAB runs of many independent replicas                                     */
/* ------------------------------------------------------------------------- */
/*
 * x, v: R x n x 3 (in/out). zm: R (in/out). step: R (in/out, global step
 * counter per replica). rep_id: R global replica ids (Philox counter word).
 * Runs n_steps steps; every save_every steps (counted by the global step),
 * writes frame x, z, z_m, E_pot and the bias functional accumulated so far into
 * the per-replica slots [R][max_frames] (n_saved returns the count per replica).
 * T_acc: R (in/out) bias functional sum_i (1/(m_i gamma)) |F_bias,i|^2 dt, summed
 * over the post-step configurations.
 */
int orc_run_baoab(const orc_ff* ff, const orc_bias* b, int R, double* x, double* v,
                  double* zm, int64_t* step, const int32_t* rep_id, uint64_t seed, double dt,
                  double gamma, double kT, int64_t n_steps, int save_every, int max_frames,
                  double* frames, double* fz, double* fzm, double* fepot, double* fT,
                  int32_t* n_saved, double* T_acc, int n_threads) {
    const int n = ff->n;
    const double c1 = exp(-gamma * dt);
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int r = 0; r < R; ++r) {
        double* xr = x + (size_t)r * n * 3;
        double* vr = v + (size_t)r * n * 3;
        double* F = (double*)malloc(sizeof(double) * 3 * (size_t)n);
        double* work = (double*)malloc(sizeof(double) * 3 * (size_t)n);
        orc_eval ev;
        int saved = 0;
        eval_all(ff, b, xr, F, work, &zm[r], &ev);
        for (int64_t s = 0; s < n_steps; ++s) {
            const uint32_t st = (uint32_t)step[r];
            for (int i = 0; i < n; ++i) {
                const double im = 1.0 / ff->mass[i];
                double xi[4];
                orc_normals4(seed, (uint32_t)i, (uint32_t)rep_id[r], st, 0u, xi);
                const double sd = sqrt((1.0 - c1 * c1) * kT * im);
                for (int k = 0; k < 3; ++k) {
                    double vv = vr[3 * i + k] + 0.5 * dt * F[3 * i + k] * im; /* B */
                    double xx = xr[3 * i + k] + 0.5 * dt * vv;                /* A */
                    vv = c1 * vv + sd * xi[k];                               /* O */
                    xx += 0.5 * dt * vv;                                     /* A */
                    vr[3 * i + k] = vv;
                    xr[3 * i + k] = xx;
                }
            }
            eval_all(ff, b, xr, F, work, &zm[r], &ev);
            for (int i = 0; i < n; ++i)
                for (int k = 0; k < 3; ++k) vr[3 * i + k] += 0.5 * dt * F[3 * i + k] / ff->mass[i]; /* B */
            step[r] += 1;
            if (T_acc) T_acc[r] += dt * ev.fbias2_over_m / gamma;
            if (save_every > 0 && step[r] % save_every == 0 && saved < max_frames) {
                const size_t slot = (size_t)r * max_frames + saved;
                if (frames) memcpy(frames + slot * n * 3, xr, sizeof(double) * 3 * (size_t)n);
                if (fz) fz[slot] = ev.z;
                if (fzm) fzm[slot] = ev.zm;
                if (fepot) fepot[slot] = ev.epot;
                if (fT) fT[slot] = T_acc ? T_acc[r] : 0.0;
                saved++;
            }
        }
        if (n_saved) n_saved[r] = saved;
        free(F);
        free(work);
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Two-dimensional toy: U = (x^2 - 1)^2 + y^2, z = (x - x_ref)^2, overdamped   */
/* ------------------------------------------------------------------------- */
static void toy_force(const double* p, double* f) {
    f[0] = -4.0 * p[0] * (p[0] * p[0] - 1.0);
    f[1] = -2.0 * p[1];
}

/* Euler-Maruyama runs of R independent particles. xy: R x 2, zm: R (in/out;
 * pass z(X0) for the paper's z_m(0) = z(X(0))), step: R. Frames every save_every
 * steps into [R][max_frames] (xy, z, z_m). */
int orc_run_toy(int R, double* xy, double* zm, int64_t* step, const int32_t* rep_id,
                uint64_t seed, double dt, double gamma, double kT, double k_R, double x_ref,
                int64_t n_steps, int save_every, int max_frames, double* frames, double* fz,
                double* fzm, int32_t* n_saved, double* T_acc) {
    const double sd = sqrt(2.0 * kT * dt / gamma);
    for (int r = 0; r < R; ++r) {
        double* p = xy + 2 * (size_t)r;
        int saved = 0;
        for (int64_t s = 0; s < n_steps; ++s) {
            double f[2], xi[4];
            toy_force(p, f);
            const double z = (p[0] - x_ref) * (p[0] - x_ref);
            const double sb = orc_ratchet(z, &zm[r], k_R);
            const double fb = sb * 2.0 * (p[0] - x_ref);
            f[0] += fb;
            if (T_acc) T_acc[r] += dt * fb * fb / gamma;
            orc_normals4(seed, 0u, (uint32_t)rep_id[r], (uint32_t)step[r], 0u, xi);
            p[0] += dt / gamma * f[0] + sd * xi[0];
            p[1] += dt / gamma * f[1] + sd * xi[1];
            step[r] += 1;
            if (save_every > 0 && step[r] % save_every == 0 && saved < max_frames) {
                const size_t slot = (size_t)r * max_frames + saved;
                const double z1 = (p[0] - x_ref) * (p[0] - x_ref);
                if (frames) {
                    frames[2 * slot] = p[0];
                    frames[2 * slot + 1] = p[1];
                }
                if (fz) fz[slot] = z1;
                if (fzm) fzm[slot] = zm[r] < z1 ? zm[r] : z1;
                saved++;
            }
        }
        if (n_saved) n_saved[r] = saved;
    }
    return 0;
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* Contact-map tube variables and the self-consistent rMD forces (chains)      */
/* ------------------------------------------------------------------------- */
/* Eq. (sX), Eq. (wX) with the average maps A_k = <C(t'_k)> in place of the
 * instantaneous ones, on the native-contact list p = (i, j):
 *   D_k = sum_p (C_p(X) - A_kp)^2 / sum_p C0_p^2,
 *   s = 1 - (1/t) sum_k t'_k e^{-lambda D_k} / sum_k e^{-lambda D_k},
 *   w = -(1/lambda) log sum_k e^{-lambda D_k};
 * forces of Eq. (Fs), Eq. (Fw): F^s = -k_s grad s (s - s_m) theta(s - s_m), F^w alike. */
typedef struct {
    int nc;
    const int32_t* pairs;  /* nc x 2 */
    const double* C0;      /* nc: native map entries (for the norm) */
    double r0;
    int K;
    const double* A;       /* K x nc average maps, slice-major */
    const double* tref;    /* K times t'_k */
    double lambda, k_s, k_w, t_path;
} orc_tube;

/* s, w and (optional, n x 3 each, overwritten) their gradients. */
void orc_tube_chain_vars(const orc_tube* tb, int n, const double* x, double* s, double* w,
                         double* grad_s, double* grad_w) {
    const int nc = tb->nc, K = tb->K;
    double n0 = 0.0;
    for (int p = 0; p < nc; ++p) n0 += tb->C0[p] * tb->C0[p];
    double* C = (double*)malloc(sizeof(double) * (size_t)(nc > 0 ? nc : 1));
    double* dC = (double*)malloc(sizeof(double) * (size_t)(nc > 0 ? nc : 1));
    double* D = (double*)malloc(sizeof(double) * (size_t)K);
    for (int p = 0; p < nc; ++p) {
        const int i = tb->pairs[2 * p], j = tb->pairs[2 * p + 1];
        double r2 = 0.0;
        for (int k = 0; k < 3; ++k) r2 += (x[3 * j + k] - x[3 * i + k]) * (x[3 * j + k] - x[3 * i + k]);
        const double u = r2 / (tb->r0 * tb->r0);
        const double num = 1.0 + u + u * u;
        C[p] = num / (num + u * u * u + u * u * u * u);
        dC[p] = contact_dC_du(u);
    }
    double dmin = INFINITY;
    for (int k = 0; k < K; ++k) {
        double d = 0.0;
        for (int p = 0; p < nc; ++p) d += (C[p] - tb->A[(size_t)k * nc + p]) * (C[p] - tb->A[(size_t)k * nc + p]);
        D[k] = d / n0;
        if (D[k] < dmin) dmin = D[k];
    }
    double Z = 0.0, Zt = 0.0;
    for (int k = 0; k < K; ++k) {
        const double e = exp(-tb->lambda * (D[k] - dmin));
        Z += e;
        Zt += tb->tref[k] * e;
    }
    const double tbar = Zt / Z;
    *s = 1.0 - tbar / tb->t_path;
    *w = dmin - log(Z) / tb->lambda;
    if (grad_s || grad_w) {
        /* dD_k/dC_p = 2 (C_p - A_kp) / n0; ds/dD_k = (lambda/t) pi_k (t'_k - tbar); dw/dD_k = pi_k */
        if (grad_s) memset(grad_s, 0, sizeof(double) * 3 * (size_t)n);
        if (grad_w) memset(grad_w, 0, sizeof(double) * 3 * (size_t)n);
        for (int p = 0; p < nc; ++p) {
            double bs = 0.0, bw = 0.0; /* ds/dC_p, dw/dC_p */
            for (int k = 0; k < K; ++k) {
                const double pi = exp(-tb->lambda * (D[k] - dmin)) / Z;
                const double dD = 2.0 * (C[p] - tb->A[(size_t)k * nc + p]) / n0;
                bs += tb->lambda / tb->t_path * pi * (tb->tref[k] - tbar) * dD;
                bw += pi * dD;
            }
            /* dC_p/dx_j = C'(u) 2 (x_j - x_i) / r0^2, x_i the negative */
            const int i = tb->pairs[2 * p], j = tb->pairs[2 * p + 1];
            for (int k = 0; k < 3; ++k) {
                const double g = dC[p] * 2.0 * (x[3 * j + k] - x[3 * i + k]) / (tb->r0 * tb->r0);
                if (grad_s) {
                    grad_s[3 * j + k] += bs * g;
                    grad_s[3 * i + k] -= bs * g;
                }
                if (grad_w) {
                    grad_w[3 * j + k] += bw * g;
                    grad_w[3 * i + k] -= bw * g;
                }
            }
        }
    }
    free(C);
    free(dC);
    free(D);
}

/* BAOAB runs with the physical forces plus F^s + F^w (same step order, noise and
 * outputs as orc_run_baoab). smw: R x 2 running minima (s_m, w_m), in/out; frames
 * record s (fz) and its running minimum (fzm). */
int orc_run_baoab_tube(const orc_ff* ff, const orc_tube* tb, int R, double* x, double* v,
                       double* smw, int64_t* step, const int32_t* rep_id, uint64_t seed,
                       double dt, double gamma, double kT, int64_t n_steps, int save_every,
                       int max_frames, double* frames, double* fz, double* fzm, double* fT,
                       int32_t* n_saved, double* T_acc) {
    const int n = ff->n;
    const double c1 = exp(-gamma * dt);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int r = 0; r < R; ++r) {
        double* xr = x + (size_t)r * n * 3;
        double* vr = v + (size_t)r * n * 3;
        double* F = (double*)malloc(sizeof(double) * 3 * (size_t)n);
        double* gs = (double*)malloc(sizeof(double) * 3 * (size_t)n);
        double* gw = (double*)malloc(sizeof(double) * 3 * (size_t)n);
        int saved = 0;
        double s = 0.0, w = 0.0, fb2 = 0.0;
        for (int64_t it = -1; it < n_steps; ++it) {
            if (it >= 0) { /* B A O A */
                const uint32_t st = (uint32_t)step[r];
                for (int i = 0; i < n; ++i) {
                    const double im = 1.0 / ff->mass[i];
                    double xi[4];
                    orc_normals4(seed, (uint32_t)i, (uint32_t)rep_id[r], st, 0u, xi);
                    const double sd = sqrt((1.0 - c1 * c1) * kT * im);
                    for (int k = 0; k < 3; ++k) {
                        double vv = vr[3 * i + k] + 0.5 * dt * F[3 * i + k] * im;
                        double xx = xr[3 * i + k] + 0.5 * dt * vv;
                        vv = c1 * vv + sd * xi[k];
                        xx += 0.5 * dt * vv;
                        vr[3 * i + k] = vv;
                        xr[3 * i + k] = xx;
                    }
                }
            }
            /* forces at the new configuration */
            double E[ORC_E_N];
            orc_forces(ff, xr, F, E);
            orc_tube_chain_vars(tb, n, xr, &s, &w, gs, gw);
            const double cs = orc_ratchet(s, &smw[2 * r], tb->k_s);
            const double cw = orc_ratchet(w, &smw[2 * r + 1], tb->k_w);
            fb2 = 0.0;
            for (int i = 0; i < n; ++i) {
                double f2 = 0.0;
                for (int k = 0; k < 3; ++k) {
                    const double fb = cs * gs[3 * i + k] + cw * gw[3 * i + k];
                    F[3 * i + k] += fb;
                    f2 += fb * fb;
                }
                fb2 += f2 / ff->mass[i];
            }
            if (it < 0) continue;
            for (int i = 0; i < n; ++i) /* B */
                for (int k = 0; k < 3; ++k) vr[3 * i + k] += 0.5 * dt * F[3 * i + k] / ff->mass[i];
            step[r] += 1;
            if (T_acc) T_acc[r] += dt * fb2 / gamma;
            if (save_every > 0 && step[r] % save_every == 0 && saved < max_frames) {
                const size_t slot = (size_t)r * max_frames + saved;
                if (frames) memcpy(frames + slot * n * 3, xr, sizeof(double) * 3 * (size_t)n);
                if (fz) fz[slot] = s;
                if (fzm) fzm[slot] = smw[2 * r];
                if (fT) fT[slot] = T_acc ? T_acc[r] : 0.0;
                saved++;
            }
        }
        if (n_saved) n_saved[r] = saved;
        free(F);
        free(gs);
        free(gw);
    }
    return 0;
}
