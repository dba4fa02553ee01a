// Two-dimensional models, the plain one-replica-per-launch form of the
// chain step, and the Philox block generator used to check the noise stream.
#include "scps_internal.h"

namespace scps {

// ---------------------------------------------------------------------------
// Two-dimensional models, one particle per replica, overdamped Langevin
// (Euler-Maruyama) in FP64; one thread per replica runs the whole launch.
//   model 0: U = (x^2 - 1)^2 + y^2 (double well)
//   model 1: the asymmetric funnel of Eq. (U) with the parameters of Table 1
// Biases (P.bias):
//   2: ratchet of Eq. (FrMD) on z = (x - x_ref)^2
//   3: ratchet on z = sqrt(x^2 + y^2), the distance from the funnel centre
//   4: tube variables s_lambda, w_lambda of a reference path <X(t'_k)> (the
//      configuration-space form used for the funnel): D_k = |X - <X(t'_k)>|^2,
//      pi_k = exp(-lambda D_k) / sum, w = -(1/lambda) log sum_k exp(-lambda D_k),
//      s = 1 - (1/t) sum_k t'_k pi_k, each with its own ratchet (forces F^w, F^s of
//      Eq. Fw and Eq. Fs; z_m of Eq. FrMD replaced by s_m and w_m)
// ---------------------------------------------------------------------------
namespace {

constexpr double kA1 = 30.0, kA2 = 20.0, kA3 = 6.0, kS1 = 1.0, kS2 = 2.0, kS3 = 0.5;
constexpr double kW = 0.03, kYm = 0.0, kXm = 1.5;

__device__ __forceinline__ double funnel_u(double x, double y) {
    const double r2 = x * x + y * y;
    const double d2 = (x - kXm) * (x - kXm) + (y - kYm) * (y - kYm);
    const double a = r2 + kS1 * kS1, b = r2 + kS2 * kS2, c = d2 + kS3 * kS3;
    return kW * kW * r2 * r2 - kA1 * kS1 * kS1 / (a * a) + kA2 * kS2 * kS2 / (b * b) -
           kA3 * kS3 * kS3 / (c * c);
}

__device__ __forceinline__ double2 funnel_f(double x, double y) {
    const double r2 = x * x + y * y;
    const double d2 = (x - kXm) * (x - kXm) + (y - kYm) * (y - kYm);
    const double a = r2 + kS1 * kS1, b = r2 + kS2 * kS2, c = d2 + kS3 * kS3;
    // -dU/dr2 for the terms in r2, -dU/dd2 for the gate term
    const double gr = -2.0 * kW * kW * r2 - 2.0 * kA1 * kS1 * kS1 / (a * a * a) +
                      2.0 * kA2 * kS2 * kS2 / (b * b * b);
    const double gd = -2.0 * kA3 * kS3 * kS3 / (c * c * c);
    return make_double2(2.0 * (gr * x + gd * (x - kXm)), 2.0 * (gr * y + gd * (y - kYm)));
}

struct Pot2 {
    double2 f;
    double u;
};

__device__ __forceinline__ Pot2 model_force(int model, double2 p) {
    Pot2 o;
    if (model == 1) {
        o.f = funnel_f(p.x, p.y);
        o.u = funnel_u(p.x, p.y);
    } else {
        o.f = make_double2(-4.0 * p.x * (p.x * p.x - 1.0), -2.0 * p.y);
        o.u = (p.x * p.x - 1.0) * (p.x * p.x - 1.0) + p.y * p.y;
    }
    return o;
}

// Tube variables at p: s, w and their gradients.
__device__ void tube_vars(const RunParams& P, double2 p, double* s, double* w, double2* gs,
                          double2* gw) {
    double dmin = 1e300;
    for (int k = 0; k < P.tube_k; ++k) {
        const double2 q = P.tube_ref[k];
        const double d = (p.x - q.x) * (p.x - q.x) + (p.y - q.y) * (p.y - q.y);
        dmin = d < dmin ? d : dmin;
    }
    // sums with the largest weight scaled to 1 (the formulas are unchanged)
    double S = 0.0, St = 0.0;
    double2 g1 = make_double2(0.0, 0.0), g2 = make_double2(0.0, 0.0);
    for (int k = 0; k < P.tube_k; ++k) {
        const double2 q = P.tube_ref[k];
        const double dx = p.x - q.x, dy = p.y - q.y;
        const double e = exp(-P.tube_lambda * (dx * dx + dy * dy - dmin));
        const double t = P.tube_time[k];
        S += e;
        St += e * t;
        g1.x += e * 2.0 * dx;  // sum e_k grad D_k
        g1.y += e * 2.0 * dy;
        g2.x += e * t * 2.0 * dx;  // sum e_k t_k grad D_k
        g2.y += e * t * 2.0 * dy;
    }
    const double tm = St / S;  // <t'> under pi
    *w = dmin - log(S) / P.tube_lambda;
    *s = 1.0 - tm / P.tube_t;
    *gw = make_double2(g1.x / S, g1.y / S);  // sum pi_k grad D_k
    const double c = P.tube_lambda / P.tube_t;
    *gs = make_double2(c * (g2.x / S - tm * g1.x / S), c * (g2.y / S - tm * g1.y / S));
}

}  // namespace

__global__ void k_toy(StateDev st, RunParams P, const uint32_t* __restrict__ rep_ids) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= P.n_replicas) return;
    double2 p = st.xy[r];
    double zm = st.zm[r], T = st.T[r];
    double sm = st.sm[r], wm = st.wm[r];
    long long step = st.step[r];
    long long ns = st.n_saved[r];
    const uint32_t id = rep_ids[r];
    const double a = P.toy_dt_over_gamma, sd = P.toy_sd, xr = P.toy_x_ref;
    double z;
    for (long long s = 0; s < P.n_steps; ++s) {
        const Pot2 pot = model_force(P.toy_model, p);
        double fx = pot.f.x, fy = pot.f.y;
        double bx = 0.0, by = 0.0;
        if (P.bias == 2 || P.bias == 3) {
            double gx, gy;
            if (P.bias == 2) {
                z = (p.x - xr) * (p.x - xr);
                gx = 2.0 * (p.x - xr);
                gy = 0.0;
            } else {
                z = sqrt(p.x * p.x + p.y * p.y);
                gx = z > 0.0 ? p.x / z : 0.0;
                gy = z > 0.0 ? p.y / z : 0.0;
            }
            double factor = 0.0;  // Eq. (FrMD) with theta(0) = 1
            if (z < zm)
                zm = z;
            else
                factor = -P.k_R * (z - zm);
            bx = factor * gx;
            by = factor * gy;
        } else if (P.bias == 4) {
            double sv, wv;
            double2 gs, gw;
            tube_vars(P, p, &sv, &wv, &gs, &gw);
            double fs = 0.0, fw = 0.0;
            if (sv < sm) sm = sv; else fs = -P.tube_ks * (sv - sm);
            if (wv < wm) wm = wv; else fw = -P.tube_kw * (wv - wm);
            bx = fs * gs.x + fw * gw.x;
            by = fs * gs.y + fw * gw.y;
            z = sv;
        }
        fx += bx;
        fy += by;
        T += a * (bx * bx + by * by);  // (dt / gamma) |F_bias|^2, unit mass
        const uint4 rb = philox4x32_10(make_uint4(0u, id, (uint32_t)step, 0u), P.key0, P.key1);
        const double2 xi = normals2_f64(rb.x, rb.y);
        p.x = p.x + a * fx + sd * xi.x;
        p.y = p.y + a * fy + sd * xi.y;
        ++step;
        if (P.save_interval > 0 && step % P.save_interval == 0) {
            const long long slot = ns % P.max_frames;
            const long long fi = (long long)r * P.max_frames + slot;
            st.frames[2 * fi] = (float)p.x;
            st.frames[2 * fi + 1] = (float)p.y;
            double z1 = 0.0, zm1 = 0.0;
            if (P.bias == 2) {
                z1 = (p.x - xr) * (p.x - xr);
                zm1 = zm < z1 ? zm : z1;
            } else if (P.bias == 3) {
                z1 = sqrt(p.x * p.x + p.y * p.y);
                zm1 = zm < z1 ? zm : z1;
            } else if (P.bias == 4) {  // frames record s_lambda and its running minimum
                double wv;
                double2 gs, gw;
                tube_vars(P, p, &z1, &wv, &gs, &gw);
                zm1 = sm < z1 ? sm : z1;
            }
            st.fz[fi] = z1;
            st.fzm[fi] = zm1;
            st.fe[fi] = model_force(P.toy_model, p).u;
            st.fT[fi] = T;
            ++ns;
        }
    }
    // z of the final configuration (s_lambda for the tube bias)
    if (P.bias == 3) {
        z = sqrt(p.x * p.x + p.y * p.y);
    } else if (P.bias == 4) {
        double wv;
        double2 gs, gw;
        tube_vars(P, p, &z, &wv, &gs, &gw);
    } else {
        z = (p.x - xr) * (p.x - xr);
    }
    st.xy[r] = p;
    st.zm[r] = zm;
    st.sm[r] = sm;
    st.wm[r] = wm;
    st.z[r] = z;
    st.T[r] = T;
    st.step[r] = step;
    st.n_saved[r] = ns;
    if (!(isfinite(p.x) && isfinite(p.y))) st.status[r] = 1;
}

// Average path of selected replicas from their frame buffers (frames k = 0 .. K-1,
// oldest first, all kept): out[k] = mean over the selection of frame k, summed in
// selection order (one thread per frame).
__global__ void k_path_average_2d(StateDev st, int max_frames, int K, const int* __restrict__ sel,
                                  int n_sel, double2* __restrict__ out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    double sx = 0.0, sy = 0.0;
    for (int q = 0; q < n_sel; ++q) {
        const long long fi = (long long)sel[q] * max_frames + k;
        sx += (double)st.frames[2 * fi];
        sy += (double)st.frames[2 * fi + 1];
    }
    out[k] = make_double2(sx / n_sel, sy / n_sel);
}

// Average contact maps of selected chain replicas (step 3 of the SCPS iteration):
// out[k][p] = mean over the selection of C_p (Eq. Cij, FP64 from the stored FP32
// frame) of saved frame k, summed in selection order; one thread per (k, p).
__global__ void k_path_average_contacts(StateDev st, const int2* __restrict__ con_ij, int nc, int n,
                                        const long long* __restrict__ frame_off, int n_sel, int K,
                                        double inv_r0sq, double* __restrict__ out) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)K * nc) return;
    const int k = (int)(idx / nc), p = (int)(idx % nc);
    const int2 ij = con_ij[p];
    double sum = 0.0;
    for (int q = 0; q < n_sel; ++q) {
        const float* fr = st.frames + 3 * (frame_off[q] + (long long)k * n);
        double d2 = 0.0;
        for (int c = 0; c < 3; ++c) {
            const double d = (double)fr[3 * ij.y + c] - (double)fr[3 * ij.x + c];
            d2 += d * d;
        }
        const double u = d2 * inv_r0sq, num = 1.0 + u + u * u;
        sum += num / (num + u * u * u + u * u * u * u);
    }
    out[idx] = sum / n_sel;
}

cudaError_t launch_path_average_contacts(const StateDev& st, const int2* con_ij, int nc, int n,
                                         const long long* frame_off, int n_sel, int K,
                                         double inv_r0sq, double* out, cudaStream_t stream) {
    const long long total = (long long)K * nc;
    k_path_average_contacts<<<(unsigned)((total + 255) / 256), 256, 0, stream>>>(
        st, con_ij, nc, n, frame_off, n_sel, K, inv_r0sq, out);
    return cudaGetLastError();
}

cudaError_t launch_path_average_2d(const StateDev& st, int max_frames, int K, const int* sel,
                                   int n_sel, double2* out, cudaStream_t stream) {
    k_path_average_2d<<<(K + 127) / 128, 128, 0, stream>>>(st, max_frames, K, sel, n_sel, out);
    return cudaGetLastError();
}

cudaError_t launch_toy(const StateDev& st, const RunParams& P, const uint32_t* rep_ids,
                       cudaStream_t stream) {
    const int threads = 128;
    k_toy<<<(P.n_replicas + threads - 1) / threads, threads, 0, stream>>>(st, P, rep_ids);
    return cudaGetLastError();
}

__global__ void k_philox(long long n, const uint4* __restrict__ ctr, uint32_t k0, uint32_t k1,
                         uint4* __restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = philox4x32_10(ctr[i], k0, k1);
}

cudaError_t launch_philox(long long n, const uint32_t* ctr, uint32_t k0, uint32_t k1,
                          uint32_t* out, cudaStream_t stream) {
    if (n <= 0) return cudaSuccess;
    const int threads = 256;
    k_philox<<<(unsigned)((n + threads - 1) / threads), threads, 0, stream>>>(
        n, (const uint4*)ctr, k0, k1, (uint4*)out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Plain form: one replica per kernel launch per step, forces accumulated with
// FP32 atomics in global memory, no CUDA graph. The physics, the noise and the
// update order match the resident form; this is the baseline it is compared to.
// ---------------------------------------------------------------------------
struct PlainBuf {
    float* F;        // 3 n: physical force
    float* Fb;       // 3 n: bias force
    double* zacc;    // z of the replica
    double* eacc;    // potential energy of the replica
    double* factor;  // ratchet factor of the current step
    double* tacc;    // sum |F_bias|^2 / m
};

__global__ void k_plain_kick_drift(float4* x, float4* v, const float* __restrict__ F,
                                   const float* __restrict__ Fb, TopoDev tp, RunParams P,
                                   uint32_t rep_id, long long step, int with_noise) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= tp.n_atoms) return;
    const int n = tp.n_atoms;
    const float im = tp.inv_m[i];
    const float hdt = P.half_dt;
    const float fx = F[i] + Fb[i], fy = F[n + i] + Fb[n + i], fz = F[2 * n + i] + Fb[2 * n + i];
    float4 vv = v[i];
    vv.x = fmaf(hdt * im, fx, vv.x);
    vv.y = fmaf(hdt * im, fy, vv.y);
    vv.z = fmaf(hdt * im, fz, vv.z);
    if (with_noise) {
        float4 xx = x[i];
        xx.x = fmaf(hdt, vv.x, xx.x);
        xx.y = fmaf(hdt, vv.y, xx.y);
        xx.z = fmaf(hdt, vv.z, xx.z);
        const uint4 rb = philox4x32_10(make_uint4((uint32_t)i, rep_id, (uint32_t)step, 0u), P.key0, P.key1);
        const float4 xi = normals4_f32(rb);
        const float sd = tp.noise_sd[i];
        vv.x = fmaf(P.c1, vv.x, sd * xi.x);
        vv.y = fmaf(P.c1, vv.y, sd * xi.y);
        vv.z = fmaf(P.c1, vv.z, sd * xi.z);
        xx.x = fmaf(hdt, vv.x, xx.x);
        xx.y = fmaf(hdt, vv.y, xx.y);
        xx.z = fmaf(hdt, vv.z, xx.z);
        x[i] = xx;
    }
    v[i] = vv;
}

template <int ELEC>
__global__ void k_plain_pairs(const float4* __restrict__ x, float* F, double* eacc, TopoDev tp,
                              RunParams P, int energy) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = tp.n_atoms;
    if (i >= n) return;
    const float4 xi = x[i];
    const float qi = tp.qs[i];
    const float2 li = tp.lj[i];
    const unsigned long long em = tp.excl[i];
    float fx = 0.f, fy = 0.f, fz = 0.f, e = 0.f;
    for (int j = i + 1; j < n; ++j) {
        const int dj = j - i + kExclWindow;
        if (dj < 2 * kExclWindow && ((em >> dj) & 1ull)) continue;
        const float4 xj = x[j];
        const float dx = xj.x - xi.x, dy = xj.y - xi.y, dz = xj.z - xi.z;
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        if (r2 >= P.pc.rc2) continue;
        const float2 lj = tp.lj[j];
        float ep = 0.f;
        float s;
        if (energy)
            s = pair_s<ELEC, true>(r2, li.x + lj.x, li.y * lj.y, qi * tp.qs[j], P.pc, &ep);
        else
            s = pair_s<ELEC, false>(r2, li.x + lj.x, li.y * lj.y, qi * tp.qs[j], P.pc, &ep);
        fx = fmaf(s, dx, fx);
        fy = fmaf(s, dy, fy);
        fz = fmaf(s, dz, fz);
        atomicAdd(&F[j], -s * dx);
        atomicAdd(&F[n + j], -s * dy);
        atomicAdd(&F[2 * n + j], -s * dz);
        e += ep;
    }
    atomicAdd(&F[i], fx);
    atomicAdd(&F[n + i], fy);
    atomicAdd(&F[2 * n + i], fz);
    if (energy) atomicAdd(eacc, (double)e);
}

__global__ void k_plain_bonded(const float4* __restrict__ x, float* F, double* eacc, TopoDev tp,
                               int energy) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = tp.n_atoms;
    if (t < tp.n_bonds) {
        const int2 ij = tp.bond_ij[t];
        const float2 par = tp.bond_par[t];
        const float4 a = x[ij.x], c = x[ij.y];
        const float dx = c.x - a.x, dy = c.y - a.y, dz = c.z - a.z;
        const float r = sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
        const float dr = r - par.x;
        const float f = par.y * dr / r;
        atomicAdd(&F[ij.x], f * dx);
        atomicAdd(&F[n + ij.x], f * dy);
        atomicAdd(&F[2 * n + ij.x], f * dz);
        atomicAdd(&F[ij.y], -f * dx);
        atomicAdd(&F[n + ij.y], -f * dy);
        atomicAdd(&F[2 * n + ij.y], -f * dz);
        if (energy) atomicAdd(eacc, 0.5 * (double)par.y * (double)dr * (double)dr);
    } else if (t < tp.n_bonds + tp.n_angles) {
        const int q = t - tp.n_bonds;
        const int4 ijk = tp.ang_ijk[q];
        const float2 par = tp.ang_par[q];
        const float4 a = x[ijk.x], b = x[ijk.y], c = x[ijk.z];
        const float ux = a.x - b.x, uy = a.y - b.y, uz = a.z - b.z;
        const float wx = c.x - b.x, wy = c.y - b.y, wz = c.z - b.z;
        const float cx = uy * wz - uz * wy, cy = uz * wx - ux * wz, cz = ux * wy - uy * wx;
        const float sn = sqrtf(fmaf(cx, cx, fmaf(cy, cy, cz * cz)));
        const float cs = fmaf(ux, wx, fmaf(uy, wy, uz * wz));
        const float ru2 = fmaf(ux, ux, fmaf(uy, uy, uz * uz));
        const float rw2 = fmaf(wx, wx, fmaf(wy, wy, wz * wz));
        const float dth = atan2f(sn, cs) - par.x;
        const float g = -par.y * dth / sn;
        const float au = cs / ru2, aw = cs / rw2;
        const float fix = g * fmaf(au, ux, -wx), fiy = g * fmaf(au, uy, -wy), fiz = g * fmaf(au, uz, -wz);
        const float fkx = g * fmaf(aw, wx, -ux), fky = g * fmaf(aw, wy, -uy), fkz = g * fmaf(aw, wz, -uz);
        atomicAdd(&F[ijk.x], fix);
        atomicAdd(&F[n + ijk.x], fiy);
        atomicAdd(&F[2 * n + ijk.x], fiz);
        atomicAdd(&F[ijk.z], fkx);
        atomicAdd(&F[n + ijk.z], fky);
        atomicAdd(&F[2 * n + ijk.z], fkz);
        atomicAdd(&F[ijk.y], -(fix + fkx));
        atomicAdd(&F[n + ijk.y], -(fiy + fky));
        atomicAdd(&F[2 * n + ijk.y], -(fiz + fkz));
        if (energy) atomicAdd(eacc, 0.5 * (double)par.y * (double)dth * (double)dth);
    }
}

// z terms in FP64 (the straightforward way), summed with FP64 atomics.
__global__ void k_plain_contacts(const float4* __restrict__ x, float* cdelta, double* zacc,
                                 TopoDev tp, RunParams P) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= tp.n_contacts) return;
    const int2 ij = tp.con_ij[c];
    const float4 a = x[ij.x], b = x[ij.y];
    const double dx = (double)b.x - a.x, dy = (double)b.y - a.y, dz = (double)b.z - a.z;
    const double u = (dx * dx + dy * dy + dz * dz) * ((double)P.inv_r0sq_ff.hi + P.inv_r0sq_ff.lo);
    const double num = 1.0 + u + u * u;
    const double C = num / (num + u * u * u + u * u * u * u);
    const float2 c0 = tp.con_C0[c];
    const double d = C - ((double)c0.x + (double)c0.y);
    cdelta[c] = (float)d;
    atomicAdd(zacc, d * d);
}

__global__ void k_plain_ratchet(double* zacc, double* zm, double* zout, double* factor,
                                RunParams P) {
    const double z = *zacc;
    *zout = z;
    double f = 0.0;
    if (z < *zm)
        *zm = z;
    else
        f = -P.k_R * (z - *zm);
    *factor = f;
}

__global__ void k_plain_bias(const float4* __restrict__ x, const float* __restrict__ cdelta,
                             const double* factor, float* Fb, TopoDev tp, RunParams P) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= tp.n_contacts) return;
    const double fac = *factor;
    if (fac == 0.0) return;
    const int n = tp.n_atoms;
    const int2 ij = tp.con_ij[c];
    const float4 a = x[ij.x], b = x[ij.y];
    const float dx = b.x - a.x, dy = b.y - a.y, dz = b.z - a.z;
    const float u = fmaf(dx, dx, fmaf(dy, dy, dz * dz)) * P.inv_r0sq;
    const float g = (float)fac * 4.0f * P.inv_r0sq * cdelta[c] * contact_dC_du(u);
    atomicAdd(&Fb[ij.y], g * dx);
    atomicAdd(&Fb[n + ij.y], g * dy);
    atomicAdd(&Fb[2 * n + ij.y], g * dz);
    atomicAdd(&Fb[ij.x], -g * dx);
    atomicAdd(&Fb[n + ij.x], -g * dy);
    atomicAdd(&Fb[2 * n + ij.x], -g * dz);
}

__global__ void k_plain_tacc(const float* __restrict__ Fb, const double* factor, double* T,
                             TopoDev tp, RunParams P) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= tp.n_atoms || *factor == 0.0) return;
    const int n = tp.n_atoms;
    const float bx = Fb[i], by = Fb[n + i], bz = Fb[2 * n + i];
    atomicAdd(T, (double)P.dt / P.gamma * (double)((bx * bx + by * by + bz * bz) * tp.inv_m[i]));
}

__global__ void k_plain_frame(const float4* __restrict__ x, StateDev st, int r, RepDev rep, int n,
                              RunParams P, const double* eacc) {
    const long long slot = st.n_saved[r] % P.max_frames;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        float* fr = st.frames + 3 * (rep.frame_off + slot * n + i);
        fr[0] = x[i].x;
        fr[1] = x[i].y;
        fr[2] = x[i].z;
    }
}

__global__ void k_plain_frame_scalars(StateDev st, int r, RunParams P, const double* eacc) {
    const long long slot = st.n_saved[r] % P.max_frames;
    const long long fi = (long long)r * P.max_frames + slot;
    st.fz[fi] = st.z[r];
    st.fzm[fi] = st.zm[r];
    st.fe[fi] = *eacc;
    st.fT[fi] = st.T[r];
    st.n_saved[r] += 1;
}

// One force evaluation (F, Fb, z, ratchet) of replica r in the plain form.
static cudaError_t plain_eval(int elec, const TopoDev& tp, const StateDev& st, int r,
                              const RepDev& rep, const RunParams& P, const PlainBuf& b,
                              bool energy, cudaStream_t s) {
    const int n = tp.n_atoms;
    float4* x = st.x + rep.atom_off;
    cudaMemsetAsync(b.F, 0, sizeof(float) * 3 * n, s);
    cudaMemsetAsync(b.Fb, 0, sizeof(float) * 3 * n, s);
    cudaMemsetAsync(b.zacc, 0, sizeof(double), s);
    cudaMemsetAsync(b.eacc, 0, sizeof(double), s);
    const int th = 128;
    const int gb = (n + th - 1) / th;
    switch (elec) {
        case ELEC_DDIEL: k_plain_pairs<ELEC_DDIEL><<<gb, th, 0, s>>>(x, b.F, b.eacc, tp, P, energy); break;
        case ELEC_RF: k_plain_pairs<ELEC_RF><<<gb, th, 0, s>>>(x, b.F, b.eacc, tp, P, energy); break;
        case ELEC_PLAIN: k_plain_pairs<ELEC_PLAIN><<<gb, th, 0, s>>>(x, b.F, b.eacc, tp, P, energy); break;
        default: k_plain_pairs<ELEC_NONE><<<gb, th, 0, s>>>(x, b.F, b.eacc, tp, P, energy); break;
    }
    const int nbt = tp.n_bonds + tp.n_angles;
    if (nbt > 0) k_plain_bonded<<<(nbt + th - 1) / th, th, 0, s>>>(x, b.F, b.eacc, tp, energy);
    if (P.bias == 1 && tp.n_contacts > 0) {
        const int gc = (tp.n_contacts + th - 1) / th;
        float* cdelta = b.Fb + 3 * n;  // scratch after Fb
        k_plain_contacts<<<gc, th, 0, s>>>(x, cdelta, b.zacc, tp, P);
        k_plain_ratchet<<<1, 1, 0, s>>>(b.zacc, st.zm + r, st.z + r, b.factor, P);
        k_plain_bias<<<gc, th, 0, s>>>(x, cdelta, b.factor, b.Fb, tp, P);
    } else {
        cudaMemsetAsync(b.factor, 0, sizeof(double), s);
    }
    return cudaGetLastError();
}

// n_steps of replica r, launched kernel by kernel on `s`.
cudaError_t plain_run_replica(int elec, const TopoDev& tp, const StateDev& st, int r,
                              const RepDev& rep, const RunParams& P, float* scratch,
                              double* dscratch, long long step0, cudaStream_t s) {
    PlainBuf b;
    const int n = tp.n_atoms;
    b.F = scratch;
    b.Fb = scratch + 3 * n;
    b.zacc = dscratch;
    b.eacc = dscratch + 1;
    b.factor = dscratch + 2;
    b.tacc = dscratch + 3;
    const int th = 128, ga = (n + th - 1) / th;
    cudaError_t e = plain_eval(elec, tp, st, r, rep, P, b, false, s);
    if (e != cudaSuccess) return e;
    long long step = step0;
    for (long long k = 0; k < P.n_steps; ++k) {
        k_plain_kick_drift<<<ga, th, 0, s>>>(st.x + rep.atom_off, st.v + rep.atom_off, b.F, b.Fb,
                                             tp, P, rep.rep_id, step, 1);
        ++step;
        const bool save = P.save_interval > 0 && step % P.save_interval == 0;
        e = plain_eval(elec, tp, st, r, rep, P, b, save, s);
        if (e != cudaSuccess) return e;
        k_plain_kick_drift<<<ga, th, 0, s>>>(st.x + rep.atom_off, st.v + rep.atom_off, b.F, b.Fb,
                                             tp, P, rep.rep_id, step, 0);
        k_plain_tacc<<<ga, th, 0, s>>>(b.Fb, b.factor, st.T + r, tp, P);
        if (save) {
            k_plain_frame<<<ga, th, 0, s>>>(st.x + rep.atom_off, st, r, rep, n, P, b.eacc);
            k_plain_frame_scalars<<<1, 1, 0, s>>>(st, r, P, b.eacc);
        }
    }
    return cudaGetLastError();
}

}  // namespace scps

namespace scps {

// C0_ij = C_ij(X_N) of Eq. (Cij) for the native-contact list, in FP64 (a
// one-time set-up), stored as float-float for the step kernels.
__global__ void k_native_map(int nc, const int2* __restrict__ pairs, const double* __restrict__ xN,
                             double inv_r0sq, float2* __restrict__ C0) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    const int2 ij = pairs[c];
    const double dx = xN[3 * ij.y] - xN[3 * ij.x];
    const double dy = xN[3 * ij.y + 1] - xN[3 * ij.x + 1];
    const double dz = xN[3 * ij.y + 2] - xN[3 * ij.x + 2];
    const double u = (dx * dx + dy * dy + dz * dz) * inv_r0sq;
    const double num = 1.0 + u + u * u;
    const double C = num / (num + u * u * u + u * u * u * u);
    const float hi = __double2float_rn(C);
    C0[c] = make_float2(hi, __double2float_rn(C - (double)hi));
}

cudaError_t launch_native_map(int nc, const int2* pairs, const double* xN, double inv_r0sq,
                              float2* C0, cudaStream_t s) {
    if (nc <= 0) return cudaSuccess;
    k_native_map<<<(nc + 127) / 128, 128, 0, s>>>(nc, pairs, xN, inv_r0sq, C0);
    return cudaGetLastError();
}

__global__ void k_add_steps(long long* step, int n, long long k) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) step[r] += k;
}

cudaError_t launch_add_steps(long long* step, int n, long long k, cudaStream_t s) {
    k_add_steps<<<(n + 127) / 128, 128, 0, s>>>(step, n, k);
    return cudaGetLastError();
}

}  // namespace scps
