// Hessian-vector products H(X_t) V_t of the physical potential, one cluster of CL
// CTAs per frame (CL = 2 splits the block rows, bonds and angles between the two
// CTAs; each then writes half of the atoms, summing its and the peer's partials). Used by
// the double backward of the energy (the gradient of sum_t |grad U(X_t)|^2 is
// sum_t 2 H(X_t) grad U(X_t); the Onsager-Machlup action of Eq. (SOM) contains (grad U)^2).
// Pairs come in items of two 8-atom blocks whose boxes lie within r_c, on quarter warps.
//
// For a pair term phi(r) with d = x_j - x_i and w = v_j - v_i:
//   (Hv)_j = phi'' (d.w) d / r^2 + (phi'/r) (w - (d.w) d / r^2),  (Hv)_i = -(Hv)_j,
// with the shifted-force phi' (the shift is linear in r, so phi'' is unchanged).
// For an angle term k/2 (theta - theta0)^2:
//   H v = k (grad theta . v) grad theta + k (theta - theta0) D_v(grad theta),
// D_v being the directional derivative along v, written out by hand below.
// Each item sums its j terms in FP32 in a fixed order (the i terms run on over the items of
// a row of blocks); those sums go to 2^-20 fixed-point partials held as three 32-bit words
// per component (32-bit shared atomics), so results are bit-reproducible.
#include <cooperative_groups.h>

#include "scps_internal.h"

namespace cg = cooperative_groups;

namespace scps {

namespace {

constexpr unsigned kFullMask = 0xffffffffu;
constexpr int kHvpSeg = 8;           // candidate blocks J per work unit
constexpr int kHvpMaxBlocks = 512;   // 8-atom blocks per frame (4096 atoms)

struct HvpShared {
    float4* xq;      // (x, y, z, qs)
    float4* vq;      // direction v
    float2* lj;
    unsigned long long* ex;  // exclusion mask per atom slot
    int* H2;         // 3 x nta: bits 40 and up of the 2^-20 fixed-point partials (signed)
    unsigned* H1;    // 3 x nta: bits 20..39
    unsigned* H0;    // 3 x nta: bits 0..19
    float4* blo;     // boxes of the 8-atom blocks
    float4* bhi;
    int nta;
};

// Adds x in 2^-20 fixed point as three 32-bit words (two 20-bit unsigned parts and the
// signed rest), so that the sums cover the range of Hessian-vector products of stiff bonds
// (|Hv| beyond 1e10) with 32-bit shared atomics; each unsigned word takes up to 4095
// additions.
__device__ __forceinline__ void hred(const HvpShared& sm, int k, float x) {
    const long long v = f2fix(x);
    atomicAdd(&sm.H0[k], (unsigned)(v & 0xfffffll));
    atomicAdd(&sm.H1[k], (unsigned)((v >> 20) & 0xfffffll));
    atomicAdd(&sm.H2[k], (int)(v >> 40));
}

__device__ __forceinline__ void hadd(const HvpShared& sm, int i, float x, float y, float z) {
    hred(sm, i, x);
    hred(sm, sm.nta + i, y);
    hred(sm, 2 * sm.nta + i, z);
}

// phi'(r)/r of the shifted-force pair potential and phi''(r).
template <int ELEC>
__device__ __forceinline__ void pair_derivs(float r2, float sig, float eps24, float qq,
                                            const PairConst& pc, float& p1, float& pp) {
    const float inv_r = rsqrtf(r2);
    const float inv_r2 = inv_r * inv_r;
    const float sig2 = sig * sig;
    const float s2 = sig2 * inv_r2;
    const float s6 = s2 * s2 * s2;
    const float s12 = s6 * s6;
    p1 = -eps24 * fmaf(2.0f, s12, -s6) * inv_r2;     // LJ phi'/r
    pp = eps24 * fmaf(26.0f, s12, -7.0f * s6) * inv_r2;  // LJ phi''
    const float c2 = sig2 * pc.inv_rc2;
    const float c6 = c2 * c2 * c2;
    const float a_ljc = eps24 * c6 * fmaf(2.0f, c6, -1.0f);
    float cc = 0.0f;
    if (ELEC == ELEC_DDIEL) {        // phi = (qq/2) / r^2
        p1 -= qq * inv_r2 * inv_r2;
        pp += 3.0f * qq * inv_r2 * inv_r2;
        cc = qq * pc.inv_rc3;
    } else if (ELEC == ELEC_RF) {    // phi = qq (1/r + krf r^2 - crf)
        p1 += qq * fmaf(-inv_r2, inv_r, 2.0f * pc.krf);
        pp += qq * fmaf(2.0f * inv_r2, inv_r, 2.0f * pc.krf);
        cc = qq * fmaf(pc.inv_rc2, 1.0f, -2.0f * pc.krf * pc.rc);
    } else if (ELEC == ELEC_PLAIN) { // phi = qq / r
        p1 -= qq * inv_r2 * inv_r;
        pp += 2.0f * qq * inv_r2 * inv_r;
        cc = qq * pc.inv_rc2;
    }
    p1 = fmaf(fmaf(a_ljc, pc.inv_rc, cc), inv_r, p1);  // phi_sf' = phi' - phi'(rc)
}

template <int ELEC>
__device__ __forceinline__ void pair_hvp_term(const HvpShared& sm, const PairConst& pc, int i, int j,
                                              const float4& xj, const float4& vj, const float2& lj,
                                              bool ok, float& ax, float& ay, float& az) {
    const float4 xi = sm.xq[i];
    const float4 vi = sm.vq[i];
    const float2 li = sm.lj[i];
    const float dx = xj.x - xi.x, dy = xj.y - xi.y, dz = xj.z - xi.z;
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    ok = ok && r2 < pc.rc2;
    float p1, pp;
    pair_derivs<ELEC>(r2, li.x + lj.x, li.y * lj.y, xi.w * xj.w, pc, p1, pp);
    const float wx = vj.x - vi.x, wy = vj.y - vi.y, wz = vj.z - vi.z;
    const float dw = fmaf(dx, wx, fmaf(dy, wy, dz * wz));
    const float c1 = (pp - p1) * dw / r2;
    ax = ok ? fmaf(c1, dx, p1 * wx) : 0.f;
    ay = ok ? fmaf(c1, dy, p1 * wy) : 0.f;
    az = ok ? fmaf(c1, dz, p1 * wz) : 0.f;
}

// The 64 pairs of block I (8 atoms) with block J >= I on a quarter warp: lane l holds atom
// j = 8 J + l; at iteration t it takes atom i = 8 I + (l ^ t), so the i sums move by one xor
// exchange per iteration (after the eighth, xor 7, lane l again holds atom 8 I + l's) while
// the j sum stays in the lane and goes to the fixed-point partials after the item. The i sums (hi*) run on over the
// items of the row. Within a block (I == J) a pair counts once (j > i). Near blocks test the
// exclusion masks. An idle quarter (live false) runs along with no terms.
template <int ELEC>
__device__ __forceinline__ void hvp_item(const HvpShared& sm, const PairConst& pc, int I, int J,
                                         int lane, bool live, float& hix, float& hiy, float& hiz) {
    const int l8 = lane & 7;
    const int j = 8 * J + l8;
    const float4 xj = sm.xq[j];
    const float4 vj = sm.vq[j];
    const float2 lj = sm.lj[j];
    const bool near = 8 * (J - I) < kExclWindow + 8;
    float hjx = 0.f, hjy = 0.f, hjz = 0.f;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const int i = (8 * I + l8) ^ t;
        bool ok = live && (I != J || j > i);
        if (near) {
            const int dj = j - i + kExclWindow;
            if (dj >= 0 && dj < 2 * kExclWindow) ok = ok && !((sm.ex[i] >> dj) & 1ull);
        }
        float ax, ay, az;
        pair_hvp_term<ELEC>(sm, pc, i, j, xj, vj, lj, ok, ax, ay, az);
        hix -= ax;
        hiy -= ay;
        hiz -= az;
        hjx += ax;
        hjy += ay;
        hjz += az;
        const int m = t < 7 ? t ^ (t + 1) : 7;  // to the lane that takes atom i next
        hix = __shfl_xor_sync(kFullMask, hix, m);
        hiy = __shfl_xor_sync(kFullMask, hiy, m);
        hiz = __shfl_xor_sync(kFullMask, hiz, m);
    }
    if (live) hadd(sm, j, hjx, hjy, hjz);
}

__device__ void hvp_bond(const HvpShared& sm, const TopoDev& tp, int b) {
    const int2 ij = tp.bond_ij[b];
    const float2 par = tp.bond_par[b];
    const float4 a = sm.xq[ij.x], c = sm.xq[ij.y];
    const float4 va = sm.vq[ij.x], vc = sm.vq[ij.y];
    const float dx = c.x - a.x, dy = c.y - a.y, dz = c.z - a.z;
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const float r = sqrtf(r2);
    const float p1 = par.y * (r - par.x) / r;  // phi'/r
    const float wx = vc.x - va.x, wy = vc.y - va.y, wz = vc.z - va.z;
    const float dw = fmaf(dx, wx, fmaf(dy, wy, dz * wz));
    const float c1 = (par.y - p1) * dw / r2;
    const float ax = fmaf(c1, dx, p1 * wx), ay = fmaf(c1, dy, p1 * wy), az = fmaf(c1, dz, p1 * wz);
    hadd(sm, ij.y, ax, ay, az);
    hadd(sm, ij.x, -ax, -ay, -az);
}

__device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
    return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float3 lin(float a, float3 x, float b, float3 y) {
    return f3(fmaf(a, x.x, b * y.x), fmaf(a, x.y, b * y.y), fmaf(a, x.z, b * y.z));
}

__device__ void hvp_angle(const HvpShared& sm, const TopoDev& tp, int q) {
    const int4 ijk = tp.ang_ijk[q];
    const float2 par = tp.ang_par[q];
    const float4 A = sm.xq[ijk.x], B = sm.xq[ijk.y], Cc = sm.xq[ijk.z];
    const float4 VA = sm.vq[ijk.x], VB = sm.vq[ijk.y], VC = sm.vq[ijk.z];
    const float3 u = f3(A.x - B.x, A.y - B.y, A.z - B.z), w = f3(Cc.x - B.x, Cc.y - B.y, Cc.z - B.z);
    const float3 du = f3(VA.x - VB.x, VA.y - VB.y, VA.z - VB.z);
    const float3 dw = f3(VC.x - VB.x, VC.y - VB.y, VC.z - VB.z);
    const float3 c = cross3(u, w);
    const float sn = sqrtf(dot3(c, c));
    const float cs = dot3(u, w);
    const float ru2 = dot3(u, u), rw2 = dot3(w, w);
    const float dth = atan2f(sn, cs) - par.x;
    // grad theta: G_i = (cs u / |u|^2 - w) / sn, G_k = (cs w / |w|^2 - u) / sn, G_j = -(G_i + G_k)
    const float isn = 1.0f / sn;
    const float3 Gi = lin(cs / ru2 * isn, u, -isn, w);
    const float3 Gk = lin(cs / rw2 * isn, w, -isn, u);
    // directional derivatives along v
    const float dcs = dot3(du, w) + dot3(u, dw);
    const float3 dc = f3(cross3(du, w).x + cross3(u, dw).x, cross3(du, w).y + cross3(u, dw).y,
                         cross3(du, w).z + cross3(u, dw).z);
    const float dsn = dot3(c, dc) * isn;
    const float dru2 = 2.0f * dot3(u, du), drw2 = 2.0f * dot3(w, dw);
    const float ai = (dcs / ru2 - cs * dru2 / (ru2 * ru2)) * isn;
    const float ak = (dcs / rw2 - cs * drw2 / (rw2 * rw2)) * isn;
    const float3 dGi = f3(ai * u.x + (cs / ru2) * isn * du.x - isn * dw.x - Gi.x * dsn * isn,
                          ai * u.y + (cs / ru2) * isn * du.y - isn * dw.y - Gi.y * dsn * isn,
                          ai * u.z + (cs / ru2) * isn * du.z - isn * dw.z - Gi.z * dsn * isn);
    const float3 dGk = f3(ak * w.x + (cs / rw2) * isn * dw.x - isn * du.x - Gk.x * dsn * isn,
                          ak * w.y + (cs / rw2) * isn * dw.y - isn * du.y - Gk.y * dsn * isn,
                          ak * w.z + (cs / rw2) * isn * dw.z - isn * du.z - Gk.z * dsn * isn);
    // grad theta . v with G_j = -(G_i + G_k): G_i.(v_i - v_j) + G_k.(v_k - v_j)
    const float gv = dot3(Gi, du) + dot3(Gk, dw);
    const float k = par.y;
    const float3 hi = lin(k * gv, Gi, k * dth, dGi);
    const float3 hk = lin(k * gv, Gk, k * dth, dGk);
    // the centre gets -(H v)_i - (H v)_k since G_j = -(G_i + G_k) and D_v G_j = -(D_v G_i + D_v G_k)
    hadd(sm, ijk.x, hi.x, hi.y, hi.z);
    hadd(sm, ijk.z, hk.x, hk.y, hk.z);
    hadd(sm, ijk.y, -(hi.x + hk.x), -(hi.y + hk.y), -(hi.z + hk.z));
}

}  // namespace

template <int CL>
__device__ __forceinline__ void hvp_cluster_sync() {
    if (CL == 1)
        __syncthreads();
    else
        cg::this_cluster().sync();
}

template <int ELEC, int CL>
__global__ void __launch_bounds__(1024)
k_hvp_frames(const TopoDev* __restrict__ topo_ptr, RunParams P, const float* __restrict__ X,
             const float* __restrict__ V, float* __restrict__ HV, int nta) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int next_row, n_units;
    __shared__ int upre[kHvpMaxBlocks];  // first work unit of each row of blocks
    const TopoDev tp = *topo_ptr;
    const int n = tp.n_atoms, nbs = nta / 8;
    HvpShared sm;
    char* p = (char*)smem_raw;
    sm.nta = nta;
    sm.xq = (float4*)p; p += sizeof(float4) * nta;
    sm.vq = (float4*)p; p += sizeof(float4) * nta;
    sm.blo = (float4*)p; p += sizeof(float4) * nbs;
    sm.bhi = (float4*)p; p += sizeof(float4) * nbs;
    sm.ex = (unsigned long long*)p; p += sizeof(unsigned long long) * nta;
    sm.H2 = (int*)p; p += sizeof(int) * 3 * nta;
    sm.H1 = (unsigned*)p; p += sizeof(unsigned) * 3 * nta;
    sm.H0 = (unsigned*)p; p += sizeof(unsigned) * 3 * nta;
    sm.lj = (float2*)p;
    const long long f = blockIdx.x / CL;
    const int rank = CL == 1 ? 0 : (int)cg::this_cluster().block_rank();
    const float* xf = X + f * n * 3;
    const float* vf = V + f * n * 3;
    for (int i = threadIdx.x; i < nta; i += blockDim.x) {
        if (i < n) {
            sm.xq[i] = make_float4(xf[3 * i], xf[3 * i + 1], xf[3 * i + 2], tp.qs[i]);
            sm.vq[i] = make_float4(vf[3 * i], vf[3 * i + 1], vf[3 * i + 2], 0.f);
            sm.lj[i] = tp.lj[i];
            sm.ex[i] = tp.excl[i];
        } else {
            sm.xq[i] = make_float4(1.0e5f * (float)(i + 1), 0.f, 0.f, 0.f);
            sm.vq[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            sm.lj[i] = make_float2(0.f, 0.f);
            sm.ex[i] = 0ull;
        }
    }
    for (int i = threadIdx.x; i < 3 * nta; i += blockDim.x) {
        sm.H2[i] = 0;
        sm.H1[i] = 0u;
        sm.H0[i] = 0u;
    }
    if (threadIdx.x == 0) next_row = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int l8 = lane & 7, q = lane >> 3;
    for (int b0 = 4 * warp; b0 < nbs; b0 += 4 * nw) {  // block boxes (valid atoms only)
        const int b = b0 + q;
        const int a = 8 * b + l8;
        const bool valid = b < nbs && a < n;
        const float4 x = valid ? sm.xq[a] : make_float4(0.f, 0.f, 0.f, 0.f);
        float lx = valid ? x.x : 3.0e38f, ly = valid ? x.y : 3.0e38f, lz = valid ? x.z : 3.0e38f;
        float hx = valid ? x.x : -3.0e38f, hy = valid ? x.y : -3.0e38f, hz = valid ? x.z : -3.0e38f;
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            lx = fminf(lx, __shfl_xor_sync(kFullMask, lx, o));
            ly = fminf(ly, __shfl_xor_sync(kFullMask, ly, o));
            lz = fminf(lz, __shfl_xor_sync(kFullMask, lz, o));
            hx = fmaxf(hx, __shfl_xor_sync(kFullMask, hx, o));
            hy = fmaxf(hy, __shfl_xor_sync(kFullMask, hy, o));
            hz = fmaxf(hz, __shfl_xor_sync(kFullMask, hz, o));
        }
        if (l8 == 0 && b < nbs) {
            sm.blo[b] = make_float4(lx, ly, lz, 0.f);
            sm.bhi[b] = make_float4(hx, hy, hz, 0.f);
        }
    }
    __syncthreads();
    const int t0 = threadIdx.x * CL + rank, tstep = blockDim.x * CL;
    for (int b = t0; b < tp.n_bonds; b += tstep) hvp_bond(sm, tp, b);
    for (int a = t0; a < tp.n_angles; a += tstep) hvp_angle(sm, tp, a);
    // work units: the rows of blocks I with I % CL == rank, each cut into segments of kHvpSeg
    // candidate blocks J >= I (long rows first); a warp pulls a unit, tests its blocks
    // against I's box and takes the hits four items at a time
    if (warp == 0) {
        int run = 0;
        for (int r0 = 0; r0 < nbs; r0 += 32) {
            const int I = r0 + lane;
            const int ns = (I < nbs && I % CL == rank) ? (nbs - I + kHvpSeg - 1) / kHvpSeg : 0;
            int x = ns;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(kFullMask, x, o);
                if (lane >= o) x += y;
            }
            if (I < nbs) upre[I] = run + x - ns;  // first unit of row I
            run += __shfl_sync(kFullMask, x, 31);
        }
        if (lane == 0) n_units = run;
    }
    __syncthreads();
    for (;;) {
        int u = 0;
        if (lane == 0) u = atomicAdd(&next_row, 1);
        u = __shfl_sync(kFullMask, u, 0);
        if (u >= n_units) break;
        int lo = 0, hi = nbs;  // the last row whose first unit is <= u
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (upre[mid] <= u) lo = mid; else hi = mid;
        }
        int I = lo;
        while (I % CL != rank) --I;  // rows of the other CTA own no units here
        const int j0 = I + kHvpSeg * (u - upre[I]);
        const float4 al = sm.blo[I], ah = sm.bhi[I];
        if (!(al.x <= ah.x)) continue;  // no atoms in block I (warp-uniform)
        const int J = j0 + lane;
        bool hit = false;
        if (lane < kHvpSeg && J < nbs) {
            const float4 bl = sm.blo[J], bh = sm.bhi[J];
            const float gx = fmaxf(0.f, fmaxf(al.x - bh.x, bl.x - ah.x));
            const float gy = fmaxf(0.f, fmaxf(al.y - bh.y, bl.y - ah.y));
            const float gz = fmaxf(0.f, fmaxf(al.z - bh.z, bl.z - ah.z));
            hit = bl.x <= bh.x && fmaf(gx, gx, fmaf(gy, gy, gz * gz)) < P.pc.rc2;
        }
        unsigned m = __ballot_sync(kFullMask, hit);
        if (!m) continue;
        float hix = 0.f, hiy = 0.f, hiz = 0.f;  // this quarter's share of atom 8 I + l8
        while (m) {
            const int nh = min(__popc(m), 4);
            unsigned mm = m;
            for (int k = 0; k < q; ++k) mm &= mm - 1u;
            const int src = __ffs(mm) - 1;
            for (int k = 0; k < nh; ++k) m &= m - 1u;
            const bool live = q < nh;
            hvp_item<ELEC>(sm, P.pc, I, live ? j0 + src : I, lane, live, hix, hiy, hiz);
        }
        // the four quarters' shares of the unit's i atoms (FP32, a fixed order)
        hix += __shfl_xor_sync(kFullMask, hix, 8);
        hiy += __shfl_xor_sync(kFullMask, hiy, 8);
        hiz += __shfl_xor_sync(kFullMask, hiz, 8);
        hix += __shfl_xor_sync(kFullMask, hix, 16);
        hiy += __shfl_xor_sync(kFullMask, hiy, 16);
        hiz += __shfl_xor_sync(kFullMask, hiz, 16);
        if (lane < 8) hadd(sm, 8 * I + lane, hix, hiy, hiz);
    }
    hvp_cluster_sync<CL>();  // every partial of the cluster is complete
    float* out = HV + f * n * 3;
    const int* o2 = CL == 1 ? sm.H2 : cg::this_cluster().map_shared_rank(sm.H2, (unsigned)(rank ^ 1));
    const unsigned* o1 = CL == 1 ? sm.H1 : cg::this_cluster().map_shared_rank(sm.H1, (unsigned)(rank ^ 1));
    const unsigned* o0 = CL == 1 ? sm.H0 : cg::this_cluster().map_shared_rank(sm.H0, (unsigned)(rank ^ 1));
    for (int i = threadIdx.x + rank * blockDim.x; i < n; i += CL * blockDim.x) {
        long long h[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int k = c * nta + i;
            h[c] = ((long long)sm.H2[k] << 40) + ((long long)sm.H1[k] << 20) + (long long)sm.H0[k];
            if (CL == 2) h[c] += ((long long)o2[k] << 40) + ((long long)o1[k] << 20) + (long long)o0[k];
        }
        out[3 * i] = fix2f(h[0]);
        out[3 * i + 1] = fix2f(h[1]);
        out[3 * i + 2] = fix2f(h[2]);
    }
    hvp_cluster_sync<CL>();  // no CTA leaves while its shared memory may still be read
}

size_t hvp_smem_bytes(int nta) {
    const int nbs = nta / 8;
    return sizeof(float4) * 2 * nta + sizeof(float4) * 2 * nbs + sizeof(unsigned long long) * nta +
           (sizeof(int) + 2 * sizeof(unsigned)) * 3 * (size_t)nta + sizeof(float2) * nta;
}

// Few frames (a checkpoint segment): a 2-CTA cluster of 1024 threads per frame, so that
// the frames spread over the SMs; many frames: one 512-thread CTA each.
template <int ELEC>
static cudaError_t launch_hvp_t(const TopoDev* topo, const RunParams& P, const float* X,
                                const float* V, float* HV, long long n_frames, int nta,
                                cudaStream_t s) {
    int dev = 0, n_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int cl = 2 * n_frames <= n_sm ? 2 : 1;
    const int threads = n_frames * cl <= n_sm ? 1024 : 512;
    const size_t smem = hvp_smem_bytes(nta);
    auto kern = cl == 2 ? k_hvp_frames<ELEC, 2> : k_hvp_frames<ELEC, 1>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(n_frames * cl));
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, kern, topo, P, X, V, HV, nta);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_hvp(int elec, const TopoDev* topo, const RunParams& P, const float* X,
                       const float* V, float* HV, long long n_frames, int nta, cudaStream_t s) {
    switch (elec) {
        case ELEC_DDIEL: return launch_hvp_t<ELEC_DDIEL>(topo, P, X, V, HV, n_frames, nta, s);
        case ELEC_RF: return launch_hvp_t<ELEC_RF>(topo, P, X, V, HV, n_frames, nta, s);
        case ELEC_PLAIN: return launch_hvp_t<ELEC_PLAIN>(topo, P, X, V, HV, n_frames, nta, s);
        default: return launch_hvp_t<ELEC_NONE>(topo, P, X, V, HV, n_frames, nta, s);
    }
}

}  // namespace scps
