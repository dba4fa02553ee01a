/* FP64 oracle of the two-dimensional models - TEST INFRASTRUCTURE ONLY.
 *
 * Follows, in the paper's order and notation:
 *   Eq. (U), Table 1 ........ the asymmetric funnel (Sec. "Diffusion in a
 *                             2-dimensional asymmetric funnel")
 *   Eq. (FrMD) .............. ratchet on z = sqrt(x^2 + y^2) (the funnel's rMD
 *                             coordinate), or on z = (x - x_ref)^2 (double well)
 *   Eq. (sX), Eq. (wX) ...... tube variables with the average path in place of the
 *                             instantaneous one (the configuration-space form the
 *                             funnel section uses): D_k = |X - <X(t'_k)>|^2,
 *                             s = 1 - (1/t) sum_k t'_k e^{-lambda D_k} / sum_k e^{-lambda D_k},
 *                             w = -(1/lambda) log sum_k e^{-lambda D_k}
 *   Eq. (Fs), Eq. (Fw) ...... F^s = -k_s grad s (s - s_m) theta(s - s_m), and F^w alike,
 *                             s_m and w_m the running minima along the trajectory
 *   Eq. (T) ................. T += dt/gamma |F^s + F^w|^2 (unit mass)
 *   overdamped Langevin ..... Euler-Maruyama, Philox4x32-10 noise as in scps_oracle.c
 * The sums over k are taken with the smallest D_k factored out of the
 * exponentials, which leaves every formula unchanged.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>

void orc_normals4(uint64_t seed, uint32_t atom, uint32_t replica, uint32_t step, uint32_t stream,
                  double out[4]);
double orc_ratchet(double z, double* zm, double k_R);

/* Table 1 */
static const double A1 = 30.0, A2 = 20.0, A3 = 6.0, S1 = 1.0, S2 = 2.0, S3 = 0.5, W = 0.03;
static const double YM = 0.0, XM = 1.5;

/* U of Eq. (U) and F = -grad U, each term differentiated on its own. */
void orc_funnel(double x, double y, double* U, double F[2]) {
    const double r2 = x * x + y * y;
    const double q1 = r2 + S1 * S1, q2 = r2 + S2 * S2;
    const double dx = x - XM, dy = y - YM;
    const double q3 = dx * dx + dy * dy + S3 * S3;
    *U = W * W * r2 * r2 - A1 * S1 * S1 / (q1 * q1) + A2 * S2 * S2 / (q2 * q2) -
         A3 * S3 * S3 / (q3 * q3);
    /* d/dx of each term */
    const double t0x = W * W * 2.0 * r2 * 2.0 * x;
    const double t1x = A1 * S1 * S1 * 2.0 * 2.0 * x / (q1 * q1 * q1);
    const double t2x = -A2 * S2 * S2 * 2.0 * 2.0 * x / (q2 * q2 * q2);
    const double t3x = A3 * S3 * S3 * 2.0 * 2.0 * dx / (q3 * q3 * q3);
    const double t0y = W * W * 2.0 * r2 * 2.0 * y;
    const double t1y = A1 * S1 * S1 * 2.0 * 2.0 * y / (q1 * q1 * q1);
    const double t2y = -A2 * S2 * S2 * 2.0 * 2.0 * y / (q2 * q2 * q2);
    const double t3y = A3 * S3 * S3 * 2.0 * 2.0 * dy / (q3 * q3 * q3);
    F[0] = -(t0x + t1x + t2x + t3x);
    F[1] = -(t0y + t1y + t2y + t3y);
}

static void double_well(double x, double y, double* U, double F[2]) {
    *U = (x * x - 1.0) * (x * x - 1.0) + y * y;
    F[0] = -4.0 * x * (x * x - 1.0);
    F[1] = -2.0 * y;
}

/* Tube variables of the point (x, y) and their gradients. */
void orc_tube_vars(int K, const double* ref, const double* tref, double lambda, double t_path,
                   double x, double y, double* s, double* w, double gs[2], double gw[2]) {
    double dmin = INFINITY;
    for (int k = 0; k < K; ++k) {
        const double d = (x - ref[2 * k]) * (x - ref[2 * k]) + (y - ref[2 * k + 1]) * (y - ref[2 * k + 1]);
        if (d < dmin) dmin = d;
    }
    double Z = 0.0, Zt = 0.0; /* sum_k e_k and sum_k t'_k e_k, e_k = e^{-lambda (D_k - dmin)} */
    for (int k = 0; k < K; ++k) {
        const double d = (x - ref[2 * k]) * (x - ref[2 * k]) + (y - ref[2 * k + 1]) * (y - ref[2 * k + 1]);
        const double e = exp(-lambda * (d - dmin));
        Z += e;
        Zt += tref[k] * e;
    }
    const double tbar = Zt / Z;
    *w = -(log(Z) - lambda * dmin) / lambda;
    *s = 1.0 - tbar / t_path;
    /* dw/dD_k = pi_k; ds/dD_k = (lambda / t) pi_k (t'_k - tbar); grad D_k = 2 (X - <X_k>) */
    gw[0] = gw[1] = gs[0] = gs[1] = 0.0;
    for (int k = 0; k < K; ++k) {
        const double ex = x - ref[2 * k], ey = y - ref[2 * k + 1];
        const double pi = exp(-lambda * (ex * ex + ey * ey - dmin)) / Z;
        const double cs = lambda / t_path * pi * (tref[k] - tbar);
        gw[0] += pi * 2.0 * ex;
        gw[1] += pi * 2.0 * ey;
        gs[0] += cs * 2.0 * ex;
        gs[1] += cs * 2.0 * ey;
    }
}

/* Euler-Maruyama runs of R particles. model: 0 double well, 1 funnel.
 * bias: 0 none, 2 z = (x - x_ref)^2, 3 z = sqrt(x^2 + y^2), 4 tube variables.
 * zm, sm, wm: running minima (in/out). Frames every save_every steps:
 * frames [R][max_frames][2], fz (z, or s for the tube bias), fzm (its minimum). */
int orc_run_2d(int model, int bias, int R, double* xy, double* zm, double* sm, double* wm,
               int64_t* step, const int32_t* rep_id, uint64_t seed, double dt, double gamma,
               double kT, double k_R, double x_ref, int K, const double* ref, const double* tref,
               double lambda, double k_s, double k_w, double t_path, int64_t n_steps,
               int save_every, int max_frames, double* frames, double* fz, double* fzm,
               int32_t* n_saved, double* T_acc) {
    const double sd = sqrt(2.0 * kT * dt / gamma);
    for (int r = 0; r < R; ++r) {
        double* p = xy + 2 * (size_t)r;
        int saved = 0;
        for (int64_t n = 0; n < n_steps; ++n) {
            double U, f[2], b[2] = {0.0, 0.0}, xi[4];
            if (model == 1)
                orc_funnel(p[0], p[1], &U, f);
            else
                double_well(p[0], p[1], &U, f);
            if (bias == 2 || bias == 3) {
                double z, g[2];
                if (bias == 2) {
                    z = (p[0] - x_ref) * (p[0] - x_ref);
                    g[0] = 2.0 * (p[0] - x_ref);
                    g[1] = 0.0;
                } else {
                    z = sqrt(p[0] * p[0] + p[1] * p[1]);
                    g[0] = z > 0.0 ? p[0] / z : 0.0;
                    g[1] = z > 0.0 ? p[1] / z : 0.0;
                }
                const double c = orc_ratchet(z, &zm[r], k_R);  /* F = c grad z */
                b[0] = c * g[0];
                b[1] = c * g[1];
            } else if (bias == 4) {
                double s, w, gs[2], gw[2];
                orc_tube_vars(K, ref, tref, lambda, t_path, p[0], p[1], &s, &w, gs, gw);
                const double cs = orc_ratchet(s, &sm[r], k_s);
                const double cw = orc_ratchet(w, &wm[r], k_w);
                b[0] = cs * gs[0] + cw * gw[0];
                b[1] = cs * gs[1] + cw * gw[1];
            }
            if (T_acc) T_acc[r] += dt / gamma * (b[0] * b[0] + b[1] * b[1]);
            orc_normals4(seed, 0u, (uint32_t)rep_id[r], (uint32_t)step[r], 0u, xi);
            p[0] += dt / gamma * (f[0] + b[0]) + sd * xi[0];
            p[1] += dt / gamma * (f[1] + b[1]) + sd * xi[1];
            step[r] += 1;
            if (save_every > 0 && step[r] % save_every == 0 && saved < max_frames) {
                const size_t slot = (size_t)r * max_frames + saved;
                double z1 = 0.0, zmin = 0.0;
                if (bias == 2 || bias == 3) {
                    z1 = bias == 2 ? (p[0] - x_ref) * (p[0] - x_ref) : sqrt(p[0] * p[0] + p[1] * p[1]);
                    zmin = zm[r] < z1 ? zm[r] : z1;
                } else if (bias == 4) {
                    double w, gs[2], gw[2];
                    orc_tube_vars(K, ref, tref, lambda, t_path, p[0], p[1], &z1, &w, gs, gw);
                    zmin = sm[r] < z1 ? sm[r] : z1;
                }
                if (frames) {
                    frames[2 * slot] = p[0];
                    frames[2 * slot + 1] = p[1];
                }
                if (fz) fz[slot] = z1;
                if (fzm) fzm[slot] = zmin;
                saved++;
            }
        }
        if (n_saved) n_saved[r] = saved;
    }
    return 0;
}
