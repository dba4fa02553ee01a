/*
 * FP64 oracle of the Hessian-vector product H(X) v of the synthetic
 * potential U (bonds, angles, shifted-force LJ + Coulomb), as needed for the
 * gradient of path-action terms built from |grad U|^2 (the Onsager-Machlup
 * action, Eq. (SOM), contains (grad U)^2).
 *
 * TEST INFRASTRUCTURE ONLY (see scps_oracle.c). H v is computed as the
 * directional derivative of grad U along v, by forward-mode differentiation:
 * every gradient expression below is evaluated on dual numbers (value,
 * tangent), so the tangent part of the result is exactly H v up to rounding.
 * The gradient expressions are restated here on duals; they follow the same
 * definitions as the plain gradient of scps_oracle.c (same potential, same
 * cutoff treatment, same exclusions).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Same layout as orc_ff in scps_oracle.c. */
typedef struct {
    int n;
    const double *mass, *charge, *sigma, *eps;
    int nb;
    const int32_t *bonds;
    const double *b0, *kb;
    int na;
    const int32_t *angles;
    const double *th0, *kth;
    int ne;
    const int32_t *excl;
    double cutoff;
    int elec;
    double k_dd;
    double eps_rf;
    double coulomb_f;
    double box;
} orc_ff_h;

typedef struct {
    double v, d;
} dn;

static dn D(double v, double d) { dn r = {v, d}; return r; }
static dn dadd(dn a, dn b) { return D(a.v + b.v, a.d + b.d); }
static dn dsub(dn a, dn b) { return D(a.v - b.v, a.d - b.d); }
static dn dmul(dn a, dn b) { return D(a.v * b.v, a.d * b.v + a.v * b.d); }
static dn ddiv(dn a, dn b) { return D(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)); }
static dn dscale(dn a, double s) { return D(a.v * s, a.d * s); }
static dn dsqrt(dn a) {
    const double s = sqrt(a.v);
    return D(s, 0.5 * a.d / s);
}
static dn datan2(dn y, dn x) {
    const double q = x.v * x.v + y.v * y.v;
    return D(atan2(y.v, x.v), (x.v * y.d - y.v * x.d) / q);
}

/* phi'(r) of the pair potential (before the shift), on duals. */
static dn pair_dphi(const orc_ff_h* ff, int i, int j, dn r) {
    const double sig = 0.5 * (ff->sigma[i] + ff->sigma[j]);
    const double eps = sqrt(ff->eps[i] * ff->eps[j]);
    const dn s = ddiv(D(sig, 0.0), r);
    const dn s2 = dmul(s, s);
    const dn s6 = dmul(dmul(s2, s2), s2);
    const dn s12 = dmul(s6, s6);
    /* LJ: -24 eps (2 s^12 - s^6) / r */
    dn out = ddiv(dscale(dsub(dscale(s12, 2.0), s6), -24.0 * eps), r);
    const double qq = ff->coulomb_f * ff->charge[i] * ff->charge[j];
    const dn r2 = dmul(r, r), r3 = dmul(r2, r);
    if (ff->elec == 1) {
        out = dadd(out, ddiv(D(-2.0 * qq / ff->k_dd, 0.0), r3));
    } else if (ff->elec == 2) {
        const double rc = ff->cutoff;
        const double krf = (ff->eps_rf - 1.0) / ((2.0 * ff->eps_rf + 1.0) * rc * rc * rc);
        out = dadd(out, dadd(ddiv(D(-qq, 0.0), r2), dscale(r, 2.0 * qq * krf)));
    } else if (ff->elec == 3) {
        out = dadd(out, ddiv(D(-qq, 0.0), r2));
    }
    return out;
}

/* grad U (value) and H v (tangent) for configuration x and direction v.
 * grad and hv are n x 3 (either may be NULL). Returns 0. */
int orc_hvp(const orc_ff_h* ff, const double* x, const double* v, double* grad, double* hv) {
    const int n = ff->n;
    dn* g = (dn*)calloc((size_t)3 * n, sizeof(dn));
    char* ex = (char*)calloc((size_t)n * n, 1);
    for (int e = 0; e < ff->ne; ++e) {
        const int a = ff->excl[2 * e], b = ff->excl[2 * e + 1];
        ex[(size_t)a * n + b] = ex[(size_t)b * n + a] = 1;
    }
#define X(a, k) D(x[3 * (a) + (k)], v[3 * (a) + (k)])
    /* bonds: U = kb/2 (r - b0)^2, dU/dx_j = kb (r - b0) d / r */
    for (int b = 0; b < ff->nb; ++b) {
        const int i = ff->bonds[2 * b], j = ff->bonds[2 * b + 1];
        dn d[3];
        for (int k = 0; k < 3; ++k) d[k] = dsub(X(j, k), X(i, k));
        const dn r = dsqrt(dadd(dadd(dmul(d[0], d[0]), dmul(d[1], d[1])), dmul(d[2], d[2])));
        const dn f = ddiv(dscale(dsub(r, D(ff->b0[b], 0.0)), ff->kb[b]), r);
        for (int k = 0; k < 3; ++k) {
            g[3 * j + k] = dadd(g[3 * j + k], dmul(f, d[k]));
            g[3 * i + k] = dsub(g[3 * i + k], dmul(f, d[k]));
        }
    }
    /* angles: U = kth/2 (th - th0)^2, grad = kth (th - th0) grad th */
    for (int a = 0; a < ff->na; ++a) {
        const int i = ff->angles[3 * a], j = ff->angles[3 * a + 1], l = ff->angles[3 * a + 2];
        dn u[3], w[3];
        for (int k = 0; k < 3; ++k) {
            u[k] = dsub(X(i, k), X(j, k));
            w[k] = dsub(X(l, k), X(j, k));
        }
        const dn ru = dsqrt(dadd(dadd(dmul(u[0], u[0]), dmul(u[1], u[1])), dmul(u[2], u[2])));
        const dn rw = dsqrt(dadd(dadd(dmul(w[0], w[0]), dmul(w[1], w[1])), dmul(w[2], w[2])));
        const dn c0 = dsub(dmul(u[1], w[2]), dmul(u[2], w[1]));
        const dn c1 = dsub(dmul(u[2], w[0]), dmul(u[0], w[2]));
        const dn c2 = dsub(dmul(u[0], w[1]), dmul(u[1], w[0]));
        const dn sn = dsqrt(dadd(dadd(dmul(c0, c0), dmul(c1, c1)), dmul(c2, c2)));
        const dn cs = dadd(dadd(dmul(u[0], w[0]), dmul(u[1], w[1])), dmul(u[2], w[2]));
        const dn th = datan2(sn, cs);
        const dn coef = dscale(dsub(th, D(ff->th0[a], 0.0)), ff->kth[a]);
        const dn rr = dmul(ru, rw);
        const dn sin_t = ddiv(sn, rr), cos_t = ddiv(cs, rr);
        for (int k = 0; k < 3; ++k) {
            const dn uh = ddiv(u[k], ru), wh = ddiv(w[k], rw);
            /* d th / d x_i = (cos th u_hat - w_hat) / (|u| sin th), same for x_l */
            const dn gi = ddiv(dsub(dmul(cos_t, uh), wh), dmul(ru, sin_t));
            const dn gl = ddiv(dsub(dmul(cos_t, wh), uh), dmul(rw, sin_t));
            g[3 * i + k] = dadd(g[3 * i + k], dmul(coef, gi));
            g[3 * l + k] = dadd(g[3 * l + k], dmul(coef, gl));
            g[3 * j + k] = dsub(g[3 * j + k], dmul(coef, dadd(gi, gl)));
        }
    }
    /* non-bonded pairs within the cutoff, shifted force: dU/dx_j = (phi'(r) - phi'(rc)) d / r */
    const double rc = ff->cutoff;
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            if (ex[(size_t)i * n + j]) continue;
            dn d[3];
            for (int k = 0; k < 3; ++k) d[k] = dsub(X(j, k), X(i, k));
            const dn r2 = dadd(dadd(dmul(d[0], d[0]), dmul(d[1], d[1])), dmul(d[2], d[2]));
            if (r2.v >= rc * rc) continue;
            const dn r = dsqrt(r2);
            const dn dphi = dsub(pair_dphi(ff, i, j, r), pair_dphi(ff, i, j, D(rc, 0.0)));
            const dn f = ddiv(dphi, r);
            for (int k = 0; k < 3; ++k) {
                g[3 * j + k] = dadd(g[3 * j + k], dmul(f, d[k]));
                g[3 * i + k] = dsub(g[3 * i + k], dmul(f, d[k]));
            }
        }
#undef X
    for (int q = 0; q < 3 * n; ++q) {
        if (grad) grad[q] = g[q].v;
        if (hv) hv[q] = g[q].d;
    }
    free(g);
    free(ex);
    return 0;
}
