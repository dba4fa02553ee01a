// Resident rMD step kernel for chain replicas, and the frame evaluator.
//
// One thread-block cluster of CL CTAs (CL = 1 or 2) owns one replica for a
// whole launch of n_steps steps. Positions, velocities and int64 fixed-point
// force partials live in shared memory; the CTAs of a cluster split the force
// work and read each other's partials through distributed shared memory.
// Every step evaluates
//   bonded terms + non-bonded pairs (32 x 32 tile pairs, skipped when their
//   bounding boxes are farther apart than the cutoff)            -grad U
//   z(X) of Eq. (zrMD) from C_ij of Eq. (Cij) in float-float     collective coordinate
//   ratchet of Eq. (FrMD) in FP64 (z < z_m: z_m = z, no bias)   bias force
//   BAOAB update with Philox4x32-10 noise (Eq. Lang)
// and writes a frame every save_interval steps. Every CTA of a cluster
// integrates all atoms of the replica with the same total force, so their
// copies of the state stay identical without being exchanged.
#include <cooperative_groups.h>

#include "scps_internal.h"

namespace cg = cooperative_groups;

namespace scps {

namespace {

constexpr unsigned kFull = 0xffffffffu;

struct Shared {
    float4* xq;         // (x, y, z, qs)
    float4* v;          // velocities
    float2* lj;         // (sigma/2, sqrt(24 eps))
    long long* Fp[2];   // 3 x nta force partials of this CTA, by parity of the evaluated step
    long long* Fb;      // 3 x nta bias-force partial of this CTA
    float4* blo;        // tile bounding boxes
    float4* bhi;
    uint32_t* tpl;      // all tile pairs (I << 16 | J), I <= J
    uint32_t* tpa;      // active tile pairs of this CTA
    float* cdelta;      // C - C0 per native contact (FP32 copy of the float-float value)
    int* flag;          // force-range flag of the current evaluation
    int nta;
};

struct Scalars {
    int tp_count;
    int status;       // replica status (identical in every CTA of a cluster)
    int bias_on;
    int flag[2];      // force-range bits raised during the evaluation of a given parity
    long long n_saved;
    double zm, z, factor, epot, T;
    ff zpart[2];      // this CTA's share of z, by parity
    double epart[2];  // this CTA's share of the potential energy, by parity
    float red_f[32];
    ff red_ff[32];
    double red_d[32];
};

__device__ __forceinline__ Shared carve(void* base, int nta, int ntp_max, int ncon_max) {
    Shared s;
    char* p = (char*)base;
    s.nta = nta;
    s.xq = (float4*)p; p += sizeof(float4) * nta;
    s.v = (float4*)p; p += sizeof(float4) * nta;
    s.Fp[0] = (long long*)p; p += sizeof(long long) * 3 * nta;
    s.Fp[1] = (long long*)p; p += sizeof(long long) * 3 * nta;
    s.Fb = (long long*)p; p += sizeof(long long) * 3 * nta;
    s.lj = (float2*)p; p += sizeof(float2) * nta;
    const int nt = nta / kTile;
    s.blo = (float4*)p; p += sizeof(float4) * nt;
    s.bhi = (float4*)p; p += sizeof(float4) * nt;
    const int ntp4 = (ntp_max + 3) & ~3;
    s.tpl = (uint32_t*)p; p += sizeof(uint32_t) * ntp4;
    s.tpa = (uint32_t*)p; p += sizeof(uint32_t) * ntp4;
    s.cdelta = (float*)p;
    s.flag = nullptr;
    return s;
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ ff warp_sum_ff(ff v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ff w;
        w.hi = __shfl_down_sync(kFull, v.hi, o);
        w.lo = __shfl_down_sync(kFull, v.lo, o);
        v = ff_add(v, w);
    }
    return v;
}

// Block reductions in a fixed order (lane tree, then warps in index order):
// the result is bit-identical from run to run. Result valid on thread 0.
__device__ ff block_sum_ff(ff v, Scalars& sc) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum_ff(v);
    if (lane == 0) sc.red_ff[w] = v;
    __syncthreads();
    ff t = {0.0f, 0.0f};
    if (w == 0) {
        t = lane < nw ? sc.red_ff[lane] : ff{0.0f, 0.0f};
        t = warp_sum_ff(t);
    }
    __syncthreads();
    return t;
}

__device__ double block_sum_d(double v, Scalars& sc) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum_d(v);
    if (lane == 0) sc.red_d[w] = v;
    __syncthreads();
    double t = 0.0;
    if (w == 0) {
        t = lane < nw ? sc.red_d[lane] : 0.0;
        t = warp_sum_d(t);
    }
    __syncthreads();
    return t;
}

__device__ float block_sum_f(float v, Scalars& sc) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum_f(v);
    if (lane == 0) sc.red_f[w] = v;
    __syncthreads();
    float t = 0.0f;
    if (w == 0) {
        t = lane < nw ? sc.red_f[lane] : 0.0f;
        t = warp_sum_f(t);
    }
    __syncthreads();
    return t;
}

// Fixed-point value of a force partial; a non-finite partial or one above
// 1e9 kJ/mol/nm raises the force-range flag (the replica is then frozen).
__device__ __forceinline__ long long f2fix_checked(float v, int* flag) {
    if (!(fabsf(v) < 262144.0f)) {
        if (!(fabsf(v) <= 1.0e9f)) atomicOr(flag, SCPS_FLAG_FORCE_RANGE);
    }
    return f2fix(v);
}

__device__ __forceinline__ void add_fix(const Shared& sm, long long* F, int i, float fx, float fy,
                                        float fz) {
    const int nta = sm.nta;
    atomicAdd((unsigned long long*)&F[i], (unsigned long long)f2fix_checked(fx, sm.flag));
    atomicAdd((unsigned long long*)&F[nta + i], (unsigned long long)f2fix_checked(fy, sm.flag));
    atomicAdd((unsigned long long*)&F[2 * nta + i], (unsigned long long)f2fix_checked(fz, sm.flag));
}

// One 32 x 32 tile pair on one warp. Lane l owns atom i = 32 I + l and, in
// turn, atom j = 32 J + ((l + t) & 31) at iteration t; the j-force
// accumulators rotate one lane per iteration so that lane l ends with slot l.
template <int ELEC, bool ENERGY>
__device__ __forceinline__ float tile_pair(const Shared& sm, long long* F, const TopoDev& tp,
                                           const PairConst& pc, int I, int J, int lane) {
    const int i = I * kTile + lane;
    const float4 xi = sm.xq[i];
    const float2 li = sm.lj[i];
    const bool near = (J - I) <= 1;
    const unsigned long long em = (near && i < tp.n_atoms) ? tp.excl[i] : 0ull;
    float fix = 0.f, fiy = 0.f, fiz = 0.f, fjx = 0.f, fjy = 0.f, fjz = 0.f, eacc = 0.f;
    const int jb = J * kTile;
#pragma unroll 4
    for (int t = 0; t < kTile; ++t) {
        const int sl = (lane + t) & (kTile - 1);
        const float4 xj = sm.xq[jb + sl];
        const float2 lj = sm.lj[jb + sl];
        const float dx = xj.x - xi.x, dy = xj.y - xi.y, dz = xj.z - xi.z;
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        bool ok = r2 < pc.rc2;
        if (I == J) ok = ok && (sl > lane);
        if (near) {
            const int dj = jb + sl - i + kExclWindow;
            if (dj >= 0 && dj < 2 * kExclWindow) ok = ok && !((em >> dj) & 1ull);
        }
        float e = 0.f;
        float s = pair_s<ELEC, ENERGY>(r2, li.x + lj.x, li.y * lj.y, xi.w * xj.w, pc, &e);
        s = ok ? s : 0.0f;
        fix = fmaf(s, dx, fix);
        fiy = fmaf(s, dy, fiy);
        fiz = fmaf(s, dz, fiz);
        fjx = fmaf(-s, dx, fjx);
        fjy = fmaf(-s, dy, fjy);
        fjz = fmaf(-s, dz, fjz);
        if (ENERGY) eacc += ok ? e : 0.0f;
        const int src = (lane + 1) & (kTile - 1);
        fjx = __shfl_sync(kFull, fjx, src);
        fjy = __shfl_sync(kFull, fjy, src);
        fjz = __shfl_sync(kFull, fjz, src);
    }
    add_fix(sm, F, i, fix, fiy, fiz);
    add_fix(sm, F, jb + lane, fjx, fjy, fjz);
    return eacc;
}

// Bonds and angles with index = rank (mod nranks), strided over the CTA.
template <bool ENERGY>
__device__ double bonded(const Shared& sm, long long* F, const TopoDev& tp, int rank, int nranks) {
    double e = 0.0;
    const int stride = blockDim.x * nranks, first = threadIdx.x * nranks + rank;
    for (int b = first; b < tp.n_bonds; b += stride) {
        const int2 ij = tp.bond_ij[b];
        const float2 par = tp.bond_par[b];
        const float4 a = sm.xq[ij.x], c = sm.xq[ij.y];
        const float dx = c.x - a.x, dy = c.y - a.y, dz = c.z - a.z;
        const float r = sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
        const float dr = r - par.x;
        const float f = par.y * dr / r;
        add_fix(sm, F, ij.x, f * dx, f * dy, f * dz);
        add_fix(sm, F, ij.y, -f * dx, -f * dy, -f * dz);
        if (ENERGY) e += 0.5 * (double)par.y * (double)dr * (double)dr;
    }
    for (int q = first; q < tp.n_angles; q += stride) {
        const int4 ijk = tp.ang_ijk[q];
        const float2 par = tp.ang_par[q];
        const float4 a = sm.xq[ijk.x], b = sm.xq[ijk.y], c = sm.xq[ijk.z];
        const float ux = a.x - b.x, uy = a.y - b.y, uz = a.z - b.z;
        const float wx = c.x - b.x, wy = c.y - b.y, wz = c.z - b.z;
        const float cx = uy * wz - uz * wy, cy = uz * wx - ux * wz, cz = ux * wy - uy * wx;
        const float sn = sqrtf(fmaf(cx, cx, fmaf(cy, cy, cz * cz)));
        const float cs = fmaf(ux, wx, fmaf(uy, wy, uz * wz));
        const float ru2 = fmaf(ux, ux, fmaf(uy, uy, uz * uz));
        const float rw2 = fmaf(wx, wx, fmaf(wy, wy, wz * wz));
        const float th = atan2f(sn, cs);
        const float dth = th - par.x;
        // F_i = g (cs u / |u|^2 - w) / sn, F_k = g (cs w / |w|^2 - u) / sn, g = -k dth
        const float g = -par.y * dth / sn;
        const float au = cs / ru2, aw = cs / rw2;
        const float fix = g * fmaf(au, ux, -wx), fiy = g * fmaf(au, uy, -wy),
                    fiz = g * fmaf(au, uz, -wz);
        const float fkx = g * fmaf(aw, wx, -ux), fky = g * fmaf(aw, wy, -uy),
                    fkz = g * fmaf(aw, wz, -uz);
        add_fix(sm, F, ijk.x, fix, fiy, fiz);
        add_fix(sm, F, ijk.z, fkx, fky, fkz);
        add_fix(sm, F, ijk.y, -(fix + fkx), -(fiy + fky), -(fiz + fkz));
        if (ENERGY) e += 0.5 * (double)par.y * (double)dth * (double)dth;
    }
    return e;
}

// Cluster helpers: CL == 1 degenerates to a plain CTA.
template <int CL>
__device__ __forceinline__ void cluster_barrier() {
    if (CL == 1)
        __syncthreads();
    else
        cg::this_cluster().sync();
}

template <int CL, class T>
__device__ __forceinline__ T* peer_ptr(T* p) {
    if (CL == 1) return nullptr;
    cg::cluster_group c = cg::this_cluster();
    return c.map_shared_rank(p, c.block_rank() ^ 1u);
}

template <int CL>
__device__ __forceinline__ int cta_rank() {
    if (CL == 1) return 0;
    return (int)cg::this_cluster().block_rank();
}

// Force evaluation of the configuration in shared memory for the step of
// parity b: this CTA's share of pairs, bonds/angles and contacts go to Fp[b];
// partial z and energy are exchanged within the cluster; every CTA applies
// the same ratchet decision; the bias gradient (when engaged) goes to Fb.
// Must be called by all threads of all CTAs of the cluster.
template <int ELEC, bool ENERGY, int CL>
__device__ void evaluate(Shared& sm, Scalars& sc, const TopoDev& tp, const RunParams& P, int b,
                         bool do_ratchet) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int n = tp.n_atoms, nt = tp.n_tiles, ntp = nt * (nt + 1) / 2;
    const int rank = cta_rank<CL>();
    long long* F = sm.Fp[b];
    sm.flag = &sc.flag[b];
    // 1. tile bounding boxes (valid atoms only)
    for (int t = warp; t < nt; t += nw) {
        int a = t * kTile + lane;
        if (a >= n) a = t * kTile;
        const float4 p = sm.xq[a];
        float lx = p.x, ly = p.y, lz = p.z, hx = p.x, hy = p.y, hz = p.z;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lx = fminf(lx, __shfl_xor_sync(kFull, lx, o));
            ly = fminf(ly, __shfl_xor_sync(kFull, ly, o));
            lz = fminf(lz, __shfl_xor_sync(kFull, lz, o));
            hx = fmaxf(hx, __shfl_xor_sync(kFull, hx, o));
            hy = fmaxf(hy, __shfl_xor_sync(kFull, hy, o));
            hz = fmaxf(hz, __shfl_xor_sync(kFull, hz, o));
        }
        if (lane == 0) {
            sm.blo[t] = make_float4(lx, ly, lz, 0.f);
            sm.bhi[t] = make_float4(hx, hy, hz, 0.f);
        }
    }
    if (tid == 0) sc.tp_count = 0;
    __syncthreads();
    // 2. this CTA's tile pairs (index = rank mod CL) whose boxes come within the cutoff
    for (int p = tid * CL + rank; p < ntp; p += blockDim.x * CL) {
        const uint32_t w = sm.tpl[p];
        const int I = (int)(w >> 16), J = (int)(w & 0xffff);
        const float4 al = sm.blo[I], ah = sm.bhi[I], bl = sm.blo[J], bh = sm.bhi[J];
        const float gx = fmaxf(0.f, fmaxf(al.x - bh.x, bl.x - ah.x));
        const float gy = fmaxf(0.f, fmaxf(al.y - bh.y, bl.y - ah.y));
        const float gz = fmaxf(0.f, fmaxf(al.z - bh.z, bl.z - ah.z));
        if (fmaf(gx, gx, fmaf(gy, gy, gz * gz)) < P.pc.rc2) sm.tpa[atomicAdd(&sc.tp_count, 1)] = w;
    }
    __syncthreads();
    // 3. non-bonded tile pairs, one per warp at a time
    double e = 0.0;
    const int ntpa = sc.tp_count;
    for (int k = warp; k < ntpa; k += nw) {
        const uint32_t w = sm.tpa[k];
        const float ep = tile_pair<ELEC, ENERGY>(sm, F, tp, P.pc, (int)(w >> 16), (int)(w & 0xffff), lane);
        if (ENERGY) e += (double)ep;
    }
    // 4. bonded terms
    e += bonded<ENERGY>(sm, F, tp, rank, CL);
    // 5. native contacts: z in float-float, C - C0 kept for the gradient pass
    ff zacc = {0.0f, 0.0f};
    if (P.bias == 1) {
        for (int c = tid * CL + rank; c < tp.n_contacts; c += blockDim.x * CL) {
            const int2 ij = tp.con_ij[c];
            const float4 a = sm.xq[ij.x], bb = sm.xq[ij.y];
            const ff r2 = ff_r2(ff_diff(bb.x, a.x), ff_diff(bb.y, a.y), ff_diff(bb.z, a.z));
            const ff u = ff_mul(r2, P.inv_r0sq_ff);
            const ff C = contact_C_ff(u);
            const float2 c0 = tp.con_C0[c];
            const ff d = ff_add(C, ff{-c0.x, -c0.y});
            zacc = ff_add(zacc, ff_sqr(d));
            sm.cdelta[c] = d.hi + d.lo;
        }
    }
    const ff zsum = block_sum_ff(zacc, sc);
    double esum = 0.0;
    if (ENERGY) esum = block_sum_d(e, sc);
    if (tid == 0) {
        sc.zpart[b] = zsum;
        sc.epart[b] = esum;
    }
    // 6. exchange within the cluster; every CTA takes the same ratchet decision
    cluster_barrier<CL>();
    if (tid == 0) {
        ff zt = sc.zpart[b];
        double et = sc.epart[b];
        int fl = sc.flag[b];
        if (CL == 2) {
            const ff zp = *peer_ptr<CL>(&sc.zpart[b]);
            const double ep = *peer_ptr<CL>(&sc.epart[b]);
            fl |= *peer_ptr<CL>(&sc.flag[b]);
            zt = rank == 0 ? ff_add(zt, zp) : ff_add(zp, zt);  // rank-0 share first
            et = rank == 0 ? et + ep : ep + et;
        }
        if (ENERGY) sc.epot = et;
        if (fl) sc.status |= SCPS_FLAG_FORCE_RANGE;
        double factor = 0.0;
        if (P.bias == 1) {
            const double z = ff_to_double(zt);
            sc.z = z;
            if (do_ratchet) {  // Eq. (FrMD) with theta(0) = 1
                if (z < sc.zm)
                    sc.zm = z;
                else
                    factor = -P.k_R * (z - sc.zm);
            }
        }
        sc.factor = factor;
        sc.bias_on = factor != 0.0;
    }
    __syncthreads();
    // 7. bias force factor * grad z (only when the ratchet is engaged)
    if (sc.bias_on) {
        for (int i = tid; i < 3 * sm.nta; i += blockDim.x) sm.Fb[i] = 0;
        __syncthreads();
        const float fac = (float)sc.factor;
        const float k = fac * 4.0f * P.inv_r0sq;  // d/dx_j (C - C0)^2 = 2 d C'(u) 2 r / r0^2
        for (int c = tid * CL + rank; c < tp.n_contacts; c += blockDim.x * CL) {
            const int2 ij = tp.con_ij[c];
            const float4 a = sm.xq[ij.x], bb = sm.xq[ij.y];
            const float dx = bb.x - a.x, dy = bb.y - a.y, dz = bb.z - a.z;
            const float u = fmaf(dx, dx, fmaf(dy, dy, dz * dz)) * P.inv_r0sq;
            const float g = k * sm.cdelta[c] * contact_dC_du(u);
            add_fix(sm, sm.Fb, ij.y, g * dx, g * dy, g * dz);
            add_fix(sm, sm.Fb, ij.x, -g * dx, -g * dy, -g * dz);
        }
        cluster_barrier<CL>();
    }
}

// Sum of this CTA's and the peer's fixed-point partials for component k of atom i.
template <int CL>
__device__ __forceinline__ float sum_fix(const long long* own, const long long* peer, int idx) {
    long long v = own[idx];
    if (CL == 2) v += peer[idx];
    return fix2f(v);
}

}  // namespace

template <int ELEC, int CL>
__global__ void __launch_bounds__(1024, 1)
k_resident(const TopoDev* __restrict__ topos, const RepDev* __restrict__ reps, StateDev st,
           RunParams P, int nta, int ntp_max, int ncon_max) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Scalars sc;
    const int r = blockIdx.x / CL;
    const int rank = cta_rank<CL>();
    const RepDev rep = reps[r];
    const TopoDev tp = topos[rep.topo];
    Shared sm = carve(smem_raw, nta, ntp_max, ncon_max);
    const int n = tp.n_atoms, nt = tp.n_tiles;
    const int tid = threadIdx.x;
    const int nta3 = 3 * nta;

    for (int i = tid; i < nta; i += blockDim.x) {
        if (i < n) {
            const float4 x = st.x[rep.atom_off + i];
            sm.xq[i] = make_float4(x.x, x.y, x.z, tp.qs[i]);
            sm.lj[i] = tp.lj[i];
            sm.v[i] = st.v[rep.atom_off + i];
        } else {  // padding: far apart from everything, no charge, no LJ
            sm.xq[i] = make_float4(1.0e5f * (float)(i + 1), 0.f, 0.f, 0.f);
            sm.lj[i] = make_float2(0.f, 0.f);
            sm.v[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    for (int i = tid; i < nta3; i += blockDim.x) {
        sm.Fp[0][i] = 0;
        sm.Fp[1][i] = 0;
        sm.Fb[i] = 0;
    }
    for (int p = tid; p < nt * (nt + 1) / 2; p += blockDim.x) {  // tile-pair table, row major
        int I = 0, row = nt, q = p;
        while (q >= row) {
            q -= row;
            ++I;
            --row;
        }
        sm.tpl[p] = ((uint32_t)I << 16) | (uint32_t)(I + q);
    }
    if (tid == 0) {
        sc.zm = st.zm[r];
        sc.z = st.z[r];
        sc.T = st.T[r];
        sc.status = st.status[r];
        sc.n_saved = st.n_saved[r];
        sc.flag[0] = 0;
        sc.flag[1] = 0;
        sc.bias_on = 0;
    }
    long long step = st.step[r];
    cluster_barrier<CL>();  // every CTA of the cluster is initialised before any remote access
    const long long* pFp[2] = {peer_ptr<CL>(sm.Fp[0]), peer_ptr<CL>(sm.Fp[1])};
    const long long* pFb = peer_ptr<CL>(sm.Fb);
    if (sc.status == 0) evaluate<ELEC, false, CL>(sm, sc, tp, P, (int)(step & 1), true);

    const float hdt = P.half_dt;
    for (long long s = 0; s < P.n_steps; ++s) {
        if (sc.status != 0) break;  // frozen replica (identical in every CTA of the cluster)
        const int b = (int)(step & 1), nb = b ^ 1;
        const long long* own = sm.Fp[b];
        const bool bias = sc.bias_on;
        // B A O A (every CTA integrates every atom)
        for (int i = tid; i < n; i += blockDim.x) {
            const float im = tp.inv_m[i];
            float fx = sum_fix<CL>(own, pFp[b], i), fy = sum_fix<CL>(own, pFp[b], nta + i),
                  fz = sum_fix<CL>(own, pFp[b], 2 * nta + i);
            if (bias) {
                fx += sum_fix<CL>(sm.Fb, pFb, i);
                fy += sum_fix<CL>(sm.Fb, pFb, nta + i);
                fz += sum_fix<CL>(sm.Fb, pFb, 2 * nta + i);
            }
            float4 v = sm.v[i];
            float4 x = sm.xq[i];
            v.x = fmaf(hdt * im, fx, v.x);
            v.y = fmaf(hdt * im, fy, v.y);
            v.z = fmaf(hdt * im, fz, v.z);
            x.x = fmaf(hdt, v.x, x.x);
            x.y = fmaf(hdt, v.y, x.y);
            x.z = fmaf(hdt, v.z, x.z);
            const uint4 rb = philox4x32_10(make_uint4((uint32_t)i, rep.rep_id, (uint32_t)step, 0u),
                                           P.key0, P.key1);
            const float4 xi = normals4_f32(rb);
            const float sd = tp.noise_sd[i];
            v.x = fmaf(P.c1, v.x, sd * xi.x);
            v.y = fmaf(P.c1, v.y, sd * xi.y);
            v.z = fmaf(P.c1, v.z, sd * xi.z);
            x.x = fmaf(hdt, v.x, x.x);
            x.y = fmaf(hdt, v.y, x.y);
            x.z = fmaf(hdt, v.z, x.z);
            if (!(isfinite(x.x) && isfinite(x.y) && isfinite(x.z) && isfinite(v.x) &&
                  isfinite(v.y) && isfinite(v.z)))
                atomicOr(&sc.status, SCPS_FLAG_NONFINITE);
            sm.v[i] = v;
            sm.xq[i] = x;
        }
        // this CTA's partials of the next evaluation start from zero
        for (int i = tid; i < nta3; i += blockDim.x) sm.Fp[nb][i] = 0;
        if (tid == 0) sc.flag[nb] = 0;
        __syncthreads();
        if (sc.status != 0) break;  // non-finite state: identical decision in every CTA
        ++step;
        const bool save = P.save_interval > 0 && (step % P.save_interval) == 0;
        if (save)
            evaluate<ELEC, true, CL>(sm, sc, tp, P, nb, true);
        else
            evaluate<ELEC, false, CL>(sm, sc, tp, P, nb, true);
        // B, and the bias functional sum_i |F_bias,i|^2 / (m_i gamma) dt
        const long long slot = sc.n_saved % P.max_frames;
        const bool bias2 = sc.bias_on;
        const long long* own2 = sm.Fp[nb];
        float tb = 0.f;
        for (int i = tid; i < n; i += blockDim.x) {
            const float im = tp.inv_m[i];
            float fx = sum_fix<CL>(own2, pFp[nb], i), fy = sum_fix<CL>(own2, pFp[nb], nta + i),
                  fz = sum_fix<CL>(own2, pFp[nb], 2 * nta + i);
            if (bias2) {
                const float bx = sum_fix<CL>(sm.Fb, pFb, i), by = sum_fix<CL>(sm.Fb, pFb, nta + i),
                            bz = sum_fix<CL>(sm.Fb, pFb, 2 * nta + i);
                tb += (bx * bx + by * by + bz * bz) * im;
                fx += bx;
                fy += by;
                fz += bz;
            }
            float4 v = sm.v[i];
            v.x = fmaf(hdt * im, fx, v.x);
            v.y = fmaf(hdt * im, fy, v.y);
            v.z = fmaf(hdt * im, fz, v.z);
            sm.v[i] = v;
            if (save && rank == 0) {
                float* fr = st.frames + 3 * (rep.frame_off + slot * n + i);
                const float4 x = sm.xq[i];
                fr[0] = x.x;
                fr[1] = x.y;
                fr[2] = x.z;
            }
        }
        if (bias2) {
            const float tsum = block_sum_f(tb, sc);
            if (tid == 0) sc.T += (double)P.dt / P.gamma * (double)tsum;
        }
        if (save) {
            __syncthreads();  // every thread has used sc.n_saved for this frame
            if (tid == 0) {
                if (rank == 0) {
                    const long long fi = (long long)r * P.max_frames + slot;
                    st.fz[fi] = sc.z;
                    st.fzm[fi] = sc.zm;
                    st.fe[fi] = sc.epot;
                    st.fT[fi] = sc.T;
                }
                sc.n_saved += 1;
            }
        }
        __syncthreads();
    }
    // write back the state (rank 0; every CTA holds the same copy)
    if (rank == 0) {
        for (int i = tid; i < n; i += blockDim.x) {
            const float4 x = sm.xq[i];
            st.x[rep.atom_off + i] = make_float4(x.x, x.y, x.z, 0.f);
            st.v[rep.atom_off + i] = sm.v[i];
        }
        if (tid == 0) {
            st.zm[r] = sc.zm;
            st.z[r] = sc.z;
            st.T[r] = sc.T;
            st.status[r] = sc.status;
            st.step[r] = step;
            st.n_saved[r] = sc.n_saved;
        }
    }
    cluster_barrier<CL>();  // no CTA leaves while its shared memory may still be read
}

// Energy, forces and z of n_frames configurations (no bias, no state); one CTA per frame.
template <int ELEC>
__global__ void __launch_bounds__(1024, 1)
k_eval_frames(const TopoDev* __restrict__ topo_ptr, RunParams P, const float* __restrict__ X,
              double* __restrict__ U, float* __restrict__ F, double* __restrict__ Z, int nta,
              int ntp_max, int ncon_max) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Scalars sc;
    const TopoDev tp = *topo_ptr;
    Shared sm = carve(smem_raw, nta, ntp_max, ncon_max);
    const int n = tp.n_atoms, nt = tp.n_tiles;
    const long long f = blockIdx.x;
    const float* xf = X + f * n * 3;
    for (int i = threadIdx.x; i < nta; i += blockDim.x) {
        if (i < n) {
            sm.xq[i] = make_float4(xf[3 * i], xf[3 * i + 1], xf[3 * i + 2], tp.qs[i]);
            sm.lj[i] = tp.lj[i];
        } else {
            sm.xq[i] = make_float4(1.0e5f * (float)(i + 1), 0.f, 0.f, 0.f);
            sm.lj[i] = make_float2(0.f, 0.f);
        }
    }
    for (int i = threadIdx.x; i < 3 * nta; i += blockDim.x) sm.Fp[0][i] = 0;
    for (int p = threadIdx.x; p < nt * (nt + 1) / 2; p += blockDim.x) {
        int I = 0, row = nt, q = p;
        while (q >= row) {
            q -= row;
            ++I;
            --row;
        }
        sm.tpl[p] = ((uint32_t)I << 16) | (uint32_t)(I + q);
    }
    if (threadIdx.x == 0) {
        sc.zm = 0.0;
        sc.z = 0.0;
        sc.status = 0;
        sc.flag[0] = 0;
    }
    __syncthreads();
    evaluate<ELEC, true, 1>(sm, sc, tp, P, 0, false);
    if (F) {
        float* ff_out = F + f * n * 3;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            ff_out[3 * i] = fix2f(sm.Fp[0][i]);
            ff_out[3 * i + 1] = fix2f(sm.Fp[0][nta + i]);
            ff_out[3 * i + 2] = fix2f(sm.Fp[0][2 * nta + i]);
        }
    }
    if (threadIdx.x == 0) {
        U[f] = sc.epot;
        if (Z) Z[f] = sc.z;
    }
}

// Shared-memory bytes of the resident kernel for tiles of nta atoms.
size_t resident_smem_bytes(int nta, int ntp_max, int ncon_max) {
    const int nt = nta / kTile;
    const size_t ntp4 = (size_t)((ntp_max + 3) & ~3);
    return sizeof(float4) * nta * 2 + sizeof(long long) * 9 * nta + sizeof(float2) * nta +
           sizeof(float4) * 2 * nt + sizeof(uint32_t) * 2 * ntp4 + sizeof(float) * ncon_max;
}

template <int ELEC, int CL>
static cudaError_t launch_resident_t(const TopoDev* topos, const RepDev* reps, const StateDev& st,
                                     const RunParams& P, int nta, int ntp_max, int ncon_max,
                                     int threads, cudaStream_t stream) {
    const size_t smem = resident_smem_bytes(nta, ntp_max, ncon_max);
    auto kern = k_resident<ELEC, CL>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(P.n_replicas * CL));
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, kern, topos, reps, st, P, nta, ntp_max, ncon_max);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <int CL>
static cudaError_t launch_resident_cl(int elec, const TopoDev* topos, const RepDev* reps,
                                      const StateDev& st, const RunParams& P, int nta, int ntp_max,
                                      int ncon_max, int threads, cudaStream_t stream) {
    switch (elec) {
        case ELEC_DDIEL: return launch_resident_t<ELEC_DDIEL, CL>(topos, reps, st, P, nta, ntp_max, ncon_max, threads, stream);
        case ELEC_RF: return launch_resident_t<ELEC_RF, CL>(topos, reps, st, P, nta, ntp_max, ncon_max, threads, stream);
        case ELEC_PLAIN: return launch_resident_t<ELEC_PLAIN, CL>(topos, reps, st, P, nta, ntp_max, ncon_max, threads, stream);
        default: return launch_resident_t<ELEC_NONE, CL>(topos, reps, st, P, nta, ntp_max, ncon_max, threads, stream);
    }
}

cudaError_t launch_resident(int elec, int cluster, const TopoDev* topos, const RepDev* reps,
                            const StateDev& st, const RunParams& P, int nta, int ntp_max,
                            int ncon_max, int threads, cudaStream_t stream) {
    if (cluster == 2)
        return launch_resident_cl<2>(elec, topos, reps, st, P, nta, ntp_max, ncon_max, threads, stream);
    return launch_resident_cl<1>(elec, topos, reps, st, P, nta, ntp_max, ncon_max, threads, stream);
}

template <int ELEC>
static cudaError_t launch_eval_t(const TopoDev* topo, const RunParams& P, const float* X,
                                 double* U, float* F, double* Z, long long n_frames, int nta,
                                 int ntp_max, int ncon_max, int threads, cudaStream_t stream) {
    const size_t smem = resident_smem_bytes(nta, ntp_max, ncon_max);
    cudaError_t e = cudaFuncSetAttribute(k_eval_frames<ELEC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_eval_frames<ELEC><<<(unsigned)n_frames, threads, smem, stream>>>(topo, P, X, U, F, Z, nta,
                                                                       ntp_max, ncon_max);
    return cudaGetLastError();
}

cudaError_t launch_eval(int elec, const TopoDev* topo, const RunParams& P, const float* X,
                        double* U, float* F, double* Z, long long n_frames, int nta, int ntp_max,
                        int ncon_max, int threads, cudaStream_t stream) {
    switch (elec) {
        case ELEC_DDIEL: return launch_eval_t<ELEC_DDIEL>(topo, P, X, U, F, Z, n_frames, nta, ntp_max, ncon_max, threads, stream);
        case ELEC_RF: return launch_eval_t<ELEC_RF>(topo, P, X, U, F, Z, n_frames, nta, ntp_max, ncon_max, threads, stream);
        case ELEC_PLAIN: return launch_eval_t<ELEC_PLAIN>(topo, P, X, U, F, Z, n_frames, nta, ntp_max, ncon_max, threads, stream);
        default: return launch_eval_t<ELEC_NONE>(topo, P, X, U, F, Z, n_frames, nta, ntp_max, ncon_max, threads, stream);
    }
}

}  // namespace scps
