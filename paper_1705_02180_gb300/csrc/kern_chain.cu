// Resident rMD step kernel for chain replicas, and the frame evaluator.
//
// One thread-block cluster of CL CTAs (CL = 1 or 2) owns one replica for a
// whole launch of n_steps steps. Positions, velocities and int64 fixed-point
// force partials live in shared memory; the CTAs of a cluster split the force
// work list between them (the warps of each CTA pull their items from a counter
// in their own shared memory) and read each other's partials through
// distributed shared memory. Every step evaluates
//   bonded terms + non-bonded pairs (32 x 16 half tile pairs, skipped when
//   their bounding boxes are farther apart than the cutoff; a tile with
//   itself in one 16-step round)                                   -grad U
//   z(X) of Eq. (zrMD) from C_ij of Eq. (Cij) in float-float     collective coordinate
//   ratchet of Eq. (FrMD) in FP64 (z < z_m: z_m = z, no bias)   bias force
//   BAOAB update with Philox4x32-10 noise (Eq. Lang)
// and writes a frame every save_interval steps. Every CTA of a cluster
// integrates all atoms of the replica with the same total force, so their
// copies of the state stay identical without being exchanged. All sums that
// several warps contribute to are fixed point, so results do not depend on
// which warp or CTA took which work item.
#include <cooperative_groups.h>

#include <algorithm>
#include <climits>

#include "scps_internal.h"

namespace cg = cooperative_groups;

namespace scps {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kChunk = 32;  // contacts / bonds / angles per work item (one per lane)
constexpr int kTubeItem = 8;  // contacts per work item of the contact-map tube passes

struct Shared {
    float4* xq;         // (x, y, z, qs)
    float4* v;          // velocities (w: 1/m)
    float4* xi;         // noise of the next O half step per atom (sd times Gaussian numbers);
                        // w: the atom's |F_bias|^2 / m of the step just closed
    float2* lj;         // (sigma/2, sqrt(24 eps))
    long long* Fp[2];   // 3 x nta force partials of this CTA, by parity of the evaluated step
    long long* Gp[2];   // 3 x nta partials of sum_p (C - C0) C'(u) (x_p - x_i) over the native
                        // contacts (i, p) this CTA evaluated, by parity (the bias gradient
                        // without its ratchet factor, which is known only once z is complete)
    float4* blo;        // tile bounding boxes, then half-tile boxes (2 per tile)
    float4* bhi;
    uint32_t* tpl;      // tile pairs at least two apart (I << 16 | J), J >= I + 2
    int* flag;          // force-range flag of the current evaluation
    int nta, nt;
};

struct Scalars {
    int work_next[2];   // this CTA's work counter, by parity of the evaluated step
    int status;         // replica status (identical in every CTA of a cluster)
    int bias_on;
    int flag[2];        // force-range bits raised during the evaluation of a given parity
    long long n_saved;
    double zm, z, factor, epot, T;
    long long red_z[2][32];  // per-warp shares of z (units of 2^-40), by parity
    long long red_e[2][32];  // per-warp shares of the potential energy (units of 2^-20)
    // contact-map tube bias
    double sm, wm;                      // running minima of s_lambda and w_lambda
    float gam_sum;                      // sum_k gamma_k
    float gam[kMaxTubeK];               // gamma_k = dF/dD_k weights of the evaluated step
    int work_next2[2];                  // counter of the second work phase, by parity
    long long red_d[2][kMaxTubeK];      // this CTA's share of sum_p (C_p - A_kp)^2 (2^-40), by parity
};

__device__ __forceinline__ Shared carve(void* base, int nta, int ntp_max, int ncon_max) {
    Shared s;
    char* p = (char*)base;
    s.nta = nta;
    s.nt = nta / kTile;
    s.xq = (float4*)p; p += sizeof(float4) * nta;
    s.v = (float4*)p; p += sizeof(float4) * nta;
    s.xi = (float4*)p; p += sizeof(float4) * nta;
    s.blo = (float4*)p; p += sizeof(float4) * 3 * s.nt;
    s.bhi = (float4*)p; p += sizeof(float4) * 3 * s.nt;
    s.Fp[0] = (long long*)p; p += sizeof(long long) * 3 * nta;
    s.Fp[1] = (long long*)p; p += sizeof(long long) * 3 * nta;
    s.Gp[0] = (long long*)p; p += sizeof(long long) * 3 * nta;
    s.Gp[1] = (long long*)p; p += sizeof(long long) * 3 * nta;
    s.lj = (float2*)p; p += sizeof(float2) * nta;
    const int ntp4 = (ntp_max + 3) & ~3;
    s.tpl = (uint32_t*)p; p += sizeof(uint32_t) * ntp4;
    s.flag = nullptr;
    return s;
}

__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    return v;
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

// Half of a 32 x 32 tile pair (j slots 16h .. 16h+15) on one warp. Lane l
// owns atom i = 32 I + l; within each 16-lane half-warp, lane l takes j slot
// 16h + ((l + t) & 15) at iteration t and the j-force accumulators rotate one
// lane per iteration, so lane l ends with slot l & 15; the two half-warps'
// shares of each j are then added with one exchange. NEAR tile pairs
// (J = I + 1) test exclusions.
template <int ELEC, bool ENERGY, bool NEAR>
__device__ __forceinline__ float half_tile(const Shared& sm, long long* F, const TopoDev& tp,
                                           const PairConst& pc, int I, int J, int h, int lane) {
    const int i = I * kTile + lane;
    const float4 xi = sm.xq[i];
    const float2 li = sm.lj[i];
    const unsigned long long em = (NEAR && i < tp.n_atoms) ? tp.excl[i] : 0ull;
    const int g16 = lane & 16, l16 = lane & 15;
    const int jb = J * kTile + 16 * h;
    float fix = 0.f, fiy = 0.f, fiz = 0.f, fjx = 0.f, fjy = 0.f, fjz = 0.f, eacc = 0.f;
#pragma unroll 4
    for (int t = 0; t < 16; ++t) {
        const int sl = (l16 + t) & 15;
        const int j = jb + sl;
        const float4 xj = sm.xq[j];
        const float2 lj = sm.lj[j];
        const float dx = xj.x - xi.x, dy = xj.y - xi.y, dz = xj.z - xi.z;
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        bool ok = r2 < pc.rc2;
        if (NEAR) {
            const int dj = j - i + kExclWindow;  // in [33, 95]: j - i in [1, 64)
            if (dj < 2 * kExclWindow) ok = ok && !((em >> dj) & 1ull);
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
        const int src = g16 | ((l16 + 1) & 15);
        fjx = __shfl_sync(kFull, fjx, src);
        fjy = __shfl_sync(kFull, fjy, src);
        fjz = __shfl_sync(kFull, fjz, src);
    }
    fjx += __shfl_xor_sync(kFull, fjx, 16);
    fjy += __shfl_xor_sync(kFull, fjy, 16);
    fjz += __shfl_xor_sync(kFull, fjz, 16);
    add_fix(sm, F, i, fix, fiy, fiz);
    if (lane < 16) add_fix(sm, F, jb + lane, fjx, fjy, fjz);
    return eacc;
}

// Two quarter items side by side, one per half-warp. A quarter item is 16 i atoms
// (half a of tile I) against 16 j atoms (half h of tile J), J >= I + 2, so no pair is
// excluded. Lane l of half-warp g takes i = 32 I_g + 16 a_g + l and, at iteration t,
// j slot (l + t) & 15 of its j half; the j-force accumulators rotate within the
// half-warp, so lane l ends with slot l. Items are coded (I << 18 | J << 2 | a << 1 | h);
// a negative code leaves its half-warp idle (it adds nothing).
template <int ELEC, bool ENERGY>
__device__ __forceinline__ float quarter_items(const Shared& sm, long long* F, const PairConst& pc,
                                               int code_a, int code_b, int lane) {
    const int code = lane < 16 ? code_a : code_b;
    const bool valid = code >= 0;
    const int c = valid ? code : 0;
    const int g16 = lane & 16, l16 = lane & 15;
    const int i = (c >> 18) * kTile + 16 * ((c >> 1) & 1) + l16;
    const int jb = ((c >> 2) & 0xffff) * kTile + 16 * (c & 1);
    const float4 xi = sm.xq[i];
    const float2 li = sm.lj[i];
    const int src = g16 | ((l16 + 1) & 15);
    float fix = 0.f, fiy = 0.f, fiz = 0.f, fjx = 0.f, fjy = 0.f, fjz = 0.f, eacc = 0.f;
#pragma unroll 4
    for (int t = 0; t < 16; ++t) {
        const int j = jb + ((l16 + t) & 15);
        const float4 xj = sm.xq[j];
        const float2 lj = sm.lj[j];
        const float dx = xj.x - xi.x, dy = xj.y - xi.y, dz = xj.z - xi.z;
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const bool ok = valid && r2 < pc.rc2;
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
        fjx = __shfl_sync(kFull, fjx, src);
        fjy = __shfl_sync(kFull, fjy, src);
        fjz = __shfl_sync(kFull, fjz, src);
    }
    if (valid) {
        add_fix(sm, F, i, fix, fiy, fiz);
        add_fix(sm, F, jb + l16, fjx, fjy, fjz);
    }
    return eacc;
}

// The 496 pairs of tile I with itself in 16 iterations of one warp: at
// iteration k lane l takes the pair (l, (l + k) & 31) (k = 16 on lanes 0..15
// only), so every pair comes exactly once. The j-force accumulators rotate one
// lane per iteration; at the end lane l holds atom (l + 17) & 31's, and one
// exchange brings each to its atom's lane.
template <int ELEC, bool ENERGY>
__device__ __forceinline__ float diag_tile(const Shared& sm, long long* F, const TopoDev& tp,
                                           const PairConst& pc, int I, int lane) {
    const int i = I * kTile + lane;
    const float4 xi = sm.xq[i];
    const float2 li = sm.lj[i];
    const unsigned long long em = i < tp.n_atoms ? tp.excl[i] : 0ull;
    float fix = 0.f, fiy = 0.f, fiz = 0.f, fjx = 0.f, fjy = 0.f, fjz = 0.f, eacc = 0.f;
    const int src = (lane + 1) & 31;
#pragma unroll 4
    for (int k = 1; k <= 16; ++k) {
        const int j = I * kTile + ((lane + k) & 31);
        const float4 xj = sm.xq[j];
        const float2 lj = sm.lj[j];
        const float dx = xj.x - xi.x, dy = xj.y - xi.y, dz = xj.z - xi.z;
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const int dj = j - i + kExclWindow;  // in [1, 63]: |j - i| < 32
        const bool ok = r2 < pc.rc2 && (k < 16 || lane < 16) && !((em >> dj) & 1ull);
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
        fjx = __shfl_sync(kFull, fjx, src);
        fjy = __shfl_sync(kFull, fjy, src);
        fjz = __shfl_sync(kFull, fjz, src);
    }
    const int back = (lane + 15) & 31;
    fjx = __shfl_sync(kFull, fjx, back);
    fjy = __shfl_sync(kFull, fjy, back);
    fjz = __shfl_sync(kFull, fjz, back);
    add_fix(sm, F, i, fix + fjx, fiy + fjy, fiz + fjz);
    return eacc;
}

template <bool ENERGY>
__device__ __forceinline__ float bond_term(const Shared& sm, long long* F, const TopoDev& tp,
                                           int b) {
    const int2 ij = tp.bond_ij[b];
    const float2 par = tp.bond_par[b];
    const float4 a = sm.xq[ij.x], c = sm.xq[ij.y];
    const float dx = c.x - a.x, dy = c.y - a.y, dz = c.z - a.z;
    const float r = sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
    const float dr = r - par.x;
    const float f = par.y * dr / r;
    add_fix(sm, F, ij.x, f * dx, f * dy, f * dz);
    add_fix(sm, F, ij.y, -f * dx, -f * dy, -f * dz);
    return ENERGY ? 0.5f * par.y * dr * dr : 0.0f;
}

template <bool ENERGY>
__device__ __forceinline__ float angle_term(const Shared& sm, long long* F, const TopoDev& tp,
                                            int q) {
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
    const float dth = atan2f(sn, cs) - par.x;
    // F_i = g (cs u / |u|^2 - w) / sn, F_k = g (cs w / |w|^2 - u) / sn, g = -k dth
    const float g = -par.y * dth / sn;
    const float au = cs / ru2, aw = cs / rw2;
    const float fix = g * fmaf(au, ux, -wx), fiy = g * fmaf(au, uy, -wy), fiz = g * fmaf(au, uz, -wz);
    const float fkx = g * fmaf(aw, wx, -ux), fky = g * fmaf(aw, wy, -uy), fkz = g * fmaf(aw, wz, -uz);
    add_fix(sm, F, ijk.x, fix, fiy, fiz);
    add_fix(sm, F, ijk.z, fkx, fky, fkz);
    add_fix(sm, F, ijk.y, -(fix + fkx), -(fiy + fky), -(fiz + fkz));
    return ENERGY ? 0.5f * par.y * dth * dth : 0.0f;
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
__device__ __forceinline__ T* rank_ptr(T* p, int rank) {
    if (CL == 1) return p;
    return cg::this_cluster().map_shared_rank(p, (unsigned)rank);
}

template <int CL>
__device__ __forceinline__ int cta_rank() {
    if (CL == 1) return 0;
    return (int)cg::this_cluster().block_rank();
}

// One native contact (i, p): (C - C0)^2 in float-float, returned as a 2^-40
// fixed-point value. h (x_p - x_i) with h = (C - C0) dC/du goes to G_i and its
// negative to G_p, so that grad_i (C - C0)^2 = -4 h (x_p - x_i) / r0^2 is
// -4 G_i / r0^2 summed over the atom's contacts (Eq. zrMD, Eq. Cij).
__device__ __forceinline__ long long contact_term(const Shared& sm, long long* G, const TopoDev& tp,
                                                  const RunParams& P, int c) {
    const int2 ij = tp.con_ij[c];
    const float4 a = sm.xq[ij.x], b = sm.xq[ij.y];
    const ff r2 = ff_r2(ff_diff(b.x, a.x), ff_diff(b.y, a.y), ff_diff(b.z, a.z));
    const ff u = ff_mul(r2, P.inv_r0sq_ff);
    const ff C = contact_C_ff(u);
    const float2 c0 = tp.con_C0[c];
    const ff d = ff_add(C, ff{-c0.x, -c0.y});
    const float h = (d.hi + d.lo) * contact_dC_du(u.hi);
    const long long gx = f2fix(h * (b.x - a.x)), gy = f2fix(h * (b.y - a.y)),
                    gz = f2fix(h * (b.z - a.z));
    const int nta = sm.nta;
    atomicAdd((unsigned long long*)&G[ij.x], (unsigned long long)gx);
    atomicAdd((unsigned long long*)&G[nta + ij.x], (unsigned long long)gy);
    atomicAdd((unsigned long long*)&G[2 * nta + ij.x], (unsigned long long)gz);
    atomicAdd((unsigned long long*)&G[ij.y], (unsigned long long)(-gx));
    atomicAdd((unsigned long long*)&G[nta + ij.y], (unsigned long long)(-gy));
    atomicAdd((unsigned long long*)&G[2 * nta + ij.y], (unsigned long long)(-gz));
    return ff2fix40(ff_sqr(d));
}

// Noise of the O half step of global step `step` for atoms 32 q .. 32 q + 31:
// sqrt((1 - c1^2) kT / m_i) times Gaussian numbers from Philox4x32-10 with
// counter (atom, replica id, step, 0).
__device__ __forceinline__ void noise_chunk(const Shared& sm, const TopoDev& tp, const RunParams& P,
                                            uint32_t rep_id, long long step, int q, int lane) {
    const int i = q * kTile + lane;
    if (i < tp.n_atoms) {
        const uint4 rb = philox4x32_10(make_uint4((uint32_t)i, rep_id, (uint32_t)step, 0u), P.key0,
                                       P.key1);
        const float4 g = normals4_f32(rb);
        const float sd = tp.noise_sd[i];
        // xyz only: w holds the atom's bias-functional term, which warp 0 may still be
        // summing while the next evaluation starts
        sm.xi[i].x = sd * g.x;
        sm.xi[i].y = sd * g.y;
        sm.xi[i].z = sd * g.z;
    }
}

// Box of 32 positions of one warp (invalid lanes hold +inf/-inf sentinels):
// lane 0 writes the tile box, lanes 0 and 16 the two half-tile boxes.
__device__ __forceinline__ void warp_boxes(const Shared& sm, int t, float4 lo, float4 hi,
                                           int lane) {
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) {
        lo.x = fminf(lo.x, __shfl_xor_sync(kFull, lo.x, o));
        lo.y = fminf(lo.y, __shfl_xor_sync(kFull, lo.y, o));
        lo.z = fminf(lo.z, __shfl_xor_sync(kFull, lo.z, o));
        hi.x = fmaxf(hi.x, __shfl_xor_sync(kFull, hi.x, o));
        hi.y = fmaxf(hi.y, __shfl_xor_sync(kFull, hi.y, o));
        hi.z = fmaxf(hi.z, __shfl_xor_sync(kFull, hi.z, o));
    }
    if (t < sm.nt && (lane & 15) == 0) {
        sm.blo[sm.nt + 2 * t + (lane >> 4)] = lo;
        sm.bhi[sm.nt + 2 * t + (lane >> 4)] = hi;
    }
    lo.x = fminf(lo.x, __shfl_xor_sync(kFull, lo.x, 16));
    lo.y = fminf(lo.y, __shfl_xor_sync(kFull, lo.y, 16));
    lo.z = fminf(lo.z, __shfl_xor_sync(kFull, lo.z, 16));
    hi.x = fmaxf(hi.x, __shfl_xor_sync(kFull, hi.x, 16));
    hi.y = fmaxf(hi.y, __shfl_xor_sync(kFull, hi.y, 16));
    hi.z = fmaxf(hi.z, __shfl_xor_sync(kFull, hi.z, 16));
    if (t < sm.nt && lane == 0) {
        sm.blo[t] = lo;
        sm.bhi[t] = hi;
    }
}

// Tile and half-tile boxes of the positions in shared memory (whole CTA).
__device__ void all_boxes(const Shared& sm, int n) {
    const int lane = threadIdx.x & 31;
    for (int base = 0; base < sm.nta; base += blockDim.x) {
        const int i = base + threadIdx.x;
        float4 lo = make_float4(3.0e38f, 3.0e38f, 3.0e38f, 0.f);
        float4 hi = make_float4(-3.0e38f, -3.0e38f, -3.0e38f, 0.f);
        if (i < n) {  // i may run past the nta-entry arrays: no load then
            lo = sm.xq[i];
            hi = lo;
        }
        warp_boxes(sm, (base >> 5) + (threadIdx.x >> 5), lo, hi, lane);
    }
}

__device__ __forceinline__ float box_gap2(float4 al, float4 ah, float4 bl, float4 bh) {
    const float gx = fmaxf(0.f, fmaxf(al.x - bh.x, bl.x - ah.x));
    const float gy = fmaxf(0.f, fmaxf(al.y - bh.y, bl.y - ah.y));
    const float gz = fmaxf(0.f, fmaxf(al.z - bh.z, bl.z - ah.z));
    return fmaf(gx, gx, fmaf(gy, gy, gz * gz));
}

// C(u) of Eq. (Cij) in FP32, u = (r / r0)^2 (the tube variables need no more).
__device__ __forceinline__ float contact_C_f32(float u) {
    const float u2 = u * u;
    const float num = 1.0f + u + u2;
    return num / (num + u2 * u + u2 * u2);
}

// Contact-map tube bias, first pass over one item of kTubeItem native contacts
// (c0 .. c0 + 7): the item's share of sum_p (C_p(X) - <C_p(t'_k)>)^2 for every
// reference slice k, added in fixed point (2^-40) to the lane's running sums dacc
// (exact integer sums: independent of which warp takes which item). Lanes 0..7
// compute C of the item's contacts; then lane l takes slices l, l + 32, ... The
// item's rows of the reference maps are contiguous (contact-major, K per row), so
// each load instruction reads consecutive slices, and the eight rows of one slice
// block are loaded before any is used.
__device__ __forceinline__ void tube_pass1(const Shared& sm, const TopoDev& tp, const RunParams& P,
                                           int c0, int lane, long long* dacc) {
    const int nq = min(kTubeItem, tp.n_contacts - c0);
    float C = 0.f;
    if (lane < nq) {
        const int2 ij = tp.con_ij[c0 + lane];
        const float4 a = sm.xq[ij.x], q = sm.xq[ij.y];
        const float dx = q.x - a.x, dy = q.y - a.y, dz = q.z - a.z;
        C = contact_C_f32(fmaf(dx, dx, fmaf(dy, dy, dz * dz)) * P.inv_r0sq);
    }
    const int K = P.tube_k;
    const float* rows = tp.tube_A + (size_t)c0 * K;
#pragma unroll
    for (int blk = 0; blk < kMaxTubeK / 32; ++blk) {
        if (blk * 32 >= K) break;
        const int k = blk * 32 + lane;
        float a[kTubeItem];
#pragma unroll
        for (int q = 0; q < kTubeItem; ++q) a[q] = (q < nq && k < K) ? __ldg(rows + q * K + k) : 0.f;
        float acc = 0.f;
#pragma unroll
        for (int q = 0; q < kTubeItem; ++q) {
            const float d = __shfl_sync(kFull, C, q) - a[q];
            acc = q < nq ? fmaf(d, d, acc) : acc;
        }
        dacc[blk] += __float2ll_rn(acc * 1099511627776.0f);  // 2^40
    }
}

// Contact-map tube bias, second pass over one item of kTubeItem contacts: with
// gamma_k the weights of the ratchet forces on the slices (dF/dD_k), the force on
// the atoms of contact p is beta_p grad C_p with beta_p = (2/N0) sum_k gamma_k
// (C_p - <C_p(t'_k)>); h = beta_p C'(u) goes to G like the z gradient (F = -2/r0^2 G).
// The dots sum_k gamma_k <C_p(t'_k)> are formed with lane l on slices l, l + 32, ...
// (coalesced rows) and reduced over the warp for the eight contacts at once: three
// exchange steps halve the values each lane holds, two more finish the sums, so lane
// L ends with the dot of contact (L >> 2) & 7. The order of every sum is fixed.
__device__ __forceinline__ void tube_pass2(const Shared& sm, const Scalars& sc, const TopoDev& tp,
                                           const RunParams& P, long long* G, int c0, int lane) {
    const int nq = min(kTubeItem, tp.n_contacts - c0);
    // the contact of lane l (l < nq; clamped elsewhere) is read first, so that its
    // latency overlaps the slice loads
    const int2 ij = tp.con_ij[c0 + min(lane, nq - 1)];
    const int K = P.tube_k;
    const float* rows = tp.tube_A + (size_t)c0 * K;
    float v[kTubeItem];
#pragma unroll
    for (int q = 0; q < kTubeItem; ++q) v[q] = 0.f;
#pragma unroll
    for (int blk = 0; blk < kMaxTubeK / 32; ++blk) {
        if (blk * 32 >= K) break;
        const int k = blk * 32 + lane;
        const float g = k < K ? sc.gam[k] : 0.f;
#pragma unroll
        for (int q = 0; q < kTubeItem; ++q) {
            const float a = (q < nq && k < K) ? __ldg(rows + q * K + k) : 0.f;
            v[q] = fmaf(g, a, v[q]);
        }
    }
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
    float w4[4], w2[2];
#pragma unroll
    for (int q = 0; q < 4; ++q)
        w4[q] = (b4 ? v[q + 4] : v[q]) + __shfl_xor_sync(kFull, b4 ? v[q] : v[q + 4], 16);
#pragma unroll
    for (int q = 0; q < 2; ++q)
        w2[q] = (b3 ? w4[q + 2] : w4[q]) + __shfl_xor_sync(kFull, b3 ? w4[q] : w4[q + 2], 8);
    float w1 = (b2 ? w2[1] : w2[0]) + __shfl_xor_sync(kFull, b2 ? w2[0] : w2[1], 4);
    w1 += __shfl_xor_sync(kFull, w1, 2);
    w1 += __shfl_xor_sync(kFull, w1, 1);
    const float dot = __shfl_sync(kFull, w1, (lane & 7) * 4);
    // every lane stays to the end (all exchanges below are full-warp); lanes >= nq
    // hold a copy of the last contact and add nothing
    const bool live = lane < nq;
    const float4 a = sm.xq[ij.x], q = sm.xq[ij.y];
    const float dx = q.x - a.x, dy = q.y - a.y, dz = q.z - a.z;
    const float u = fmaf(dx, dx, fmaf(dy, dy, dz * dz)) * P.inv_r0sq;
    const float C = contact_C_f32(u);
    const float h = live ? 2.0f * tp.tube_inv_n0 * (C * sc.gam_sum - dot) * contact_dC_du(u) : 0.f;
    const long long gx = f2fix(h * dx), gy = f2fix(h * dy), gz = f2fix(h * dz);
    const int nta = sm.nta;
    if (live) {
        atomicAdd((unsigned long long*)&G[ij.x], (unsigned long long)gx);
        atomicAdd((unsigned long long*)&G[nta + ij.x], (unsigned long long)gy);
        atomicAdd((unsigned long long*)&G[2 * nta + ij.x], (unsigned long long)gz);
        atomicAdd((unsigned long long*)&G[ij.y], (unsigned long long)(-gx));
        atomicAdd((unsigned long long*)&G[nta + ij.y], (unsigned long long)(-gy));
        atomicAdd((unsigned long long*)&G[2 * nta + ij.y], (unsigned long long)(-gz));
    }
}

// Tube variables and their ratchets from the summed slice distances (warp 0):
// D_k = sum_p (C_p - <C_p(t'_k)>)^2 / N0, pi_k = exp(-lambda D_k) / sum,
// w = -(1/lambda) log sum_k exp(-lambda D_k), s = 1 - (1/t) sum_k t'_k pi_k
// (Eq. sX, Eq. wX with the average maps); F^s, F^w of Eq. (Fs), Eq. (Fw) through
// gamma_k = c_s ds/dD_k + c_w dw/dD_k, ds/dD_k = (lambda/t) pi_k (t'_k - <t'>),
// dw/dD_k = pi_k. The D_k are exact fixed-point sums; their differences to the
// smallest are taken in integers and the weights in FP32 (the FP64 pipe of this GPU
// is 64 times slower); s and w are compared with their running minima in FP64.
// Sums over k are in a fixed order (lane order, then a fixed tree).
template <int CL>
__device__ void tube_decide(Scalars& sc, const TopoDev& tp, const RunParams& P, int b, int lane) {
    const int K = P.tube_k;
    constexpr int NB = kMaxTubeK / 32;
    float tk[NB];  // slice times, loaded first (their latency overlaps the exchange)
    long long dk[NB];
    long long dmin = LLONG_MAX;
#pragma unroll
    for (int blk = 0; blk < NB; ++blk) {
        const int k = blk * 32 + lane;
        tk[blk] = k < K ? (float)P.tube_time[k] : 0.f;
        dk[blk] = LLONG_MAX;
        if (k < K) {
            long long t = 0;
            for (int q = 0; q < CL; ++q) t += rank_ptr<CL>(&sc.red_d[b][0], q)[k];
            dk[blk] = t;
            dmin = min(dmin, t);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dmin = min(dmin, __shfl_xor_sync(kFull, dmin, o));
    const float scale = 9.094947017729282e-13f * tp.tube_inv_n0;  // 2^-40 / N0
    const float lam = (float)P.tube_lambda;
    float e[NB], Z = 0.f, Zt = 0.f;
#pragma unroll
    for (int blk = 0; blk < NB; ++blk) {
        const int k = blk * 32 + lane;
        e[blk] = k < K ? expf(-lam * ((float)(dk[blk] - dmin) * scale)) : 0.f;
        Z += e[blk];
        Zt += e[blk] * tk[blk];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        Z += __shfl_down_sync(kFull, Z, o);
        Zt += __shfl_down_sync(kFull, Zt, o);
    }
    Z = __shfl_sync(kFull, Z, 0);
    Zt = __shfl_sync(kFull, Zt, 0);
    const float inv_Z = 1.0f / Z;
    const float tbar = Zt * inv_Z;
    const float inv_t = (float)(1.0 / P.tube_t);
    const double sv = 1.0 - (double)(tbar * inv_t);
    const double wv = (double)dmin * 9.094947017729282e-13 * (double)tp.tube_inv_n0 -
                      (double)(logf(Z) / lam);
    double cs = 0.0, cw = 0.0;  // ratchets, theta(0) = 1
    const double sm0 = sc.sm, wm0 = sc.wm;
    if (!(sv < sm0)) cs = -P.tube_ks * (sv - sm0);
    if (!(wv < wm0)) cw = -P.tube_kw * (wv - wm0);
    const float cs_l = (float)cs * lam * inv_t, cw_f = (float)cw;
    float gsum = 0.f;
#pragma unroll
    for (int blk = 0; blk < NB; ++blk) {
        const int k = blk * 32 + lane;
        if (k < K) {
            const float pi = e[blk] * inv_Z;
            const float g = fmaf(cs_l * pi, tk[blk] - tbar, cw_f * pi);
            sc.gam[k] = g;
            gsum += g;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) gsum += __shfl_down_sync(kFull, gsum, o);
    __syncwarp();
    if (lane == 0) {
        if (sv < sm0) sc.sm = sv;
        if (wv < wm0) sc.wm = wv;
        sc.gam_sum = gsum;
        sc.z = sv;  // frames record s_lambda and its running minimum
        sc.zm = fmin(sm0, sv);
        sc.factor = 0.5;  // the update's F = -4 factor / r0^2 G is then -2/r0^2 G
        sc.bias_on = (cs != 0.0 || cw != 0.0) ? 1 : 0;
    }
}

// Summed fixed-point partials (this CTA + peer) of one atom: force and bias gradient.
struct AtomSums {
    long long f[3], g[3];
};

// Loads the summed partials of atom i for parity b (the peer's through distributed
// shared memory); all loads are issued before any sum is formed.
template <int CL>
__device__ __forceinline__ void load_sums(const Shared& sm, int b, int peer, int i, bool bias,
                                          AtomSums& a) {
    const int nta = sm.nta;
    const long long* F = sm.Fp[b];
    const long long* G = sm.Gp[b];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        a.f[c] = F[c * nta + i];
        a.g[c] = bias ? G[c * nta + i] : 0;
    }
    if (CL == 2) {
        const long long* pF = rank_ptr<CL>(sm.Fp[b], peer);
        const long long* pG = rank_ptr<CL>(sm.Gp[b], peer);
        long long r[3], q[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            r[c] = pF[c * nta + i];
            q[c] = bias ? pG[c * nta + i] : 0;
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            a.f[c] += r[c];
            a.g[c] += q[c];
        }
    }
}

// Force evaluation of the configuration in shared memory (boxes current) for
// the evaluated step of parity b. Work items come from the queue of the
// cluster; this CTA's share goes to Fp[b] and Gp[b]; the ratchet decision is
// taken by every CTA from the same fixed-point sums. With noise_step >= 0 the
// CTA also draws the Gaussian numbers of that step's O half step for all atoms
// (each CTA of a cluster integrates every atom). On return the CTA is
// synchronised.
template <int ELEC, bool ENERGY, int CL, bool TUBE>
__device__ void evaluate(Shared& sm, Scalars& sc, const TopoDev& tp, const RunParams& P, int b,
                         bool do_ratchet, uint32_t rep_id, long long noise_step) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int nt = tp.n_tiles;
    long long* F = sm.Fp[b];
    long long* G = sm.Gp[b];
    sm.flag = &sc.flag[b];
    if (noise_step >= 0)
        for (int q = warp; q < nt; q += nw) noise_chunk(sm, tp, P, rep_id, noise_step, q, lane);
    // Work list: the pair items, then contact, bond and angle chunks. Pair items are
    // the tile pairs at least two tiles apart (far pairs), then each tile with itself,
    // then the two halves (16 j atoms) of each tile's neighbour. A warp that pulls a
    // far pair tests its four quarter items (16 x 16 atoms) by their half boxes and
    // runs the live ones two at a time, one per half-warp; an odd one waits for the
    // warp's next live quarter, or runs alone once the warp has pulled past the last
    // far pair. A neighbour half whose box is beyond the cutoff from the i tile's box
    // is skipped. Item k belongs to CTA k mod CL of the cluster, whose warps pull their
    // items from a counter in their own shared memory.
    // Under the contact-map tube bias the contact items are first-pass items of
    // kTubeItem contacts (loads from the reference maps in L2), interleaved two by two
    // with the pair items so that their memory latency overlaps arithmetic; the
    // interleave keeps every pair item on the CTA it has without the bias.
    const int nfar = nt >= 3 ? (nt - 1) * (nt - 2) / 2 : 0;
    const int n_pair = nfar + nt + 2 * (nt - 1);
    const bool tube = TUBE && do_ratchet;  // contact-map tube bias: two work phases
    const int ncon = (P.bias == 1 || P.bias == 5) ? tp.n_contacts : 0;  // frames: z too
    const int n_citems = tube ? (ncon + kTubeItem - 1) / kTubeItem : (ncon + kChunk - 1) / kChunk;
    const int m_mix = tube ? (min(n_pair, n_citems) & ~1) : 0;
    const int e_con = n_pair + n_citems;
    // one past the list position of the last far pair
    const int k_far_end = nfar == 0 ? 0
                          : 1 + (nfar - 1 < m_mix ? 4 * ((nfar - 1) >> 1) + 2 + ((nfar - 1) & 1)
                                                  : m_mix + (nfar - 1));
    const int e_bond = e_con + (tp.n_bonds + kChunk - 1) / kChunk;
    const int e_all = e_bond + (tp.n_angles + kChunk - 1) / kChunk;
    int* counter = &sc.work_next[b];
    const int rank = cta_rank<CL>();
    long long e = 0, zacc = 0;  // fixed point: sums independent of the work order
    long long dacc[TUBE ? kMaxTubeK / 32 : 1];  // first-pass slice sums of this lane
#pragma unroll
    for (int q = 0; q < (TUBE ? kMaxTubeK / 32 : 1); ++q) dacc[q] = 0;
    int pending = -1;  // code of a live quarter item waiting for a partner (warp-uniform)
    for (;;) {
        int m = 0;
        if (lane == 0) m = atomicAdd(counter, 1);
        const int k = __shfl_sync(kFull, m, 0) * CL + rank;
        if (pending >= 0 && k >= k_far_end) {  // no far pair is left for this warp
            const float ep = quarter_items<ELEC, ENERGY>(sm, F, P.pc, pending, -1, lane);
            if (ENERGY) e += f2fix(ep);
            pending = -1;
        }
        if (k >= e_all) break;
        int kp = k, kc = -1;  // pair-item index, or contact-item index when kc >= 0
        if (k < e_con) {
            if (k < 2 * m_mix) {
                const int base = (k >> 2) * 2, r4 = k & 3;
                if (r4 < 2)
                    kc = base + r4;
                else
                    kp = base + r4 - 2;
            } else {
                const int j = k - 2 * m_mix;
                if (j < n_pair - m_mix)
                    kp = m_mix + j;
                else
                    kc = m_mix + j - (n_pair - m_mix);
            }
        }
        if (k < e_con && kc < 0) {
            float ep = 0.f;
            if (kp < nfar) {
                const uint32_t w = sm.tpl[kp];
                const int I = (int)(w >> 16), J = (int)(w & 0xffff);
                bool live = false;  // lane q < 4 tests quarter (a, h) = (q >> 1, q & 1)
                if (lane < 4) {
                    const int ia = sm.nt + 2 * I + (lane >> 1), jh = sm.nt + 2 * J + (lane & 1);
                    live = box_gap2(sm.blo[ia], sm.bhi[ia], sm.blo[jh], sm.bhi[jh]) < P.pc.rc2;
                }
                unsigned lm = __ballot_sync(kFull, live);
                while (lm) {
                    const int code = (I << 18) | (J << 2) | (__ffs(lm) - 1);
                    lm &= lm - 1;
                    if (pending < 0) {
                        pending = code;
                    } else {  // each pass's energy in fixed point: the pairing is order-dependent
                        const float eq = quarter_items<ELEC, ENERGY>(sm, F, P.pc, pending, code, lane);
                        if (ENERGY) e += f2fix(eq);
                        pending = -1;
                    }
                }
            } else if (kp < nfar + nt) {
                ep = diag_tile<ELEC, ENERGY>(sm, F, tp, P.pc, kp - nfar, lane);
            } else {
                const int r = kp - nfar - nt, I = r >> 1, h = r & 1;
                const int jh = sm.nt + 2 * (I + 1) + h;  // half boxes follow sm.nt tile boxes
                if (box_gap2(sm.blo[I], sm.bhi[I], sm.blo[jh], sm.bhi[jh]) < P.pc.rc2)
                    ep = half_tile<ELEC, ENERGY, true>(sm, F, tp, P.pc, I, I + 1, h, lane);
            }
            if (ENERGY) e += f2fix(ep);
        } else if (k < e_con) {
            if (tube) {
                if constexpr (TUBE) tube_pass1(sm, tp, P, kc * kTubeItem, lane, dacc);
            } else {
                const int c0 = kc * kChunk;
                if (c0 + lane < ncon) zacc += contact_term(sm, G, tp, P, c0 + lane);
            }
        } else if (k < e_bond) {
            const int q = (k - e_con) * kChunk + lane;
            if (q < tp.n_bonds) {
                const float eb = bond_term<ENERGY>(sm, F, tp, q);
                if (ENERGY) e += f2fix(eb);
            }
        } else {
            const int q = (k - e_bond) * kChunk + lane;
            if (q < tp.n_angles) {
                const float ea = angle_term<ENERGY>(sm, F, tp, q);
                if (ENERGY) e += f2fix(ea);
            }
        }
    }
    if constexpr (TUBE) {
        if (tube) {  // one add per slice and warp into this CTA's share
#pragma unroll
            for (int blk = 0; blk < kMaxTubeK / 32; ++blk) {
                const int kk = blk * 32 + lane;
                if (kk < P.tube_k && dacc[blk] != 0)
                    atomicAdd((unsigned long long*)&sc.red_d[b][kk], (unsigned long long)dacc[blk]);
            }
        }
    }
    zacc = warp_sum_ll(zacc);
    if (ENERGY) e = warp_sum_ll(e);
    if (lane == 0) {
        sc.red_z[b][warp] = zacc;
        sc.red_e[b][warp] = e;
    }
    cluster_barrier<CL>();
    // the partials of the other parity were last read (here and in the peer CTA)
    // before this barrier: clear them for the next evaluation meanwhile
    for (int i = tid; i < 3 * sm.nta; i += blockDim.x) {
        sm.Fp[b ^ 1][i] = 0;
        sm.Gp[b ^ 1][i] = 0;
    }
    if (tube)
        for (int i = tid; i < P.tube_k; i += blockDim.x) sc.red_d[b ^ 1][i] = 0;
    // shares of z, energy and flags from every CTA of the cluster (integer sums)
    if (warp == 0) {
        long long zt = 0, et = 0;
        int fl = 0;
        for (int q = 0; q < CL; ++q) {
            if (lane < nw) {
                zt += rank_ptr<CL>(&sc.red_z[b][0], q)[lane];
                if (ENERGY) et += rank_ptr<CL>(&sc.red_e[b][0], q)[lane];
            }
            if (lane == 0) fl |= *rank_ptr<CL>(&sc.flag[b], q);
        }
        zt = warp_sum_ll(zt);
        if (ENERGY) et = warp_sum_ll(et);
        if (lane == 0) {
            if (ENERGY) sc.epot = (double)et * 9.5367431640625e-07;  // 2^-20
            if (fl) sc.status |= SCPS_FLAG_FORCE_RANGE;
            double factor = 0.0;
            if (P.bias == 1 || (P.bias == 5 && !tube)) {  // (frame evaluation: z as well)
                const double z = (double)zt * 9.094947017729282e-13;  // 2^-40
                sc.z = z;
                if (do_ratchet && P.bias == 1) {  // Eq. (FrMD) with theta(0) = 1
                    if (z < sc.zm)
                        sc.zm = z;
                    else
                        factor = -P.k_R * (z - sc.zm);
                }
            }
            sc.factor = factor;
            sc.bias_on = factor != 0.0;
            sc.work_next[b] = 0;  // every pull of this evaluation is done
        }
        if (tube) tube_decide<CL>(sc, tp, P, b, lane);
    }
    __syncthreads();
    if (tube) {  // second work phase: the bias force per contact, then G is complete
        int* counter2 = &sc.work_next2[b];
        const int n2 = (ncon + kTubeItem - 1) / kTubeItem;
        for (;;) {
            int m = 0;
            if (lane == 0) m = atomicAdd(counter2, 1);
            const int k = __shfl_sync(kFull, m, 0) * CL + rank;
            if (k >= n2) break;
            tube_pass2(sm, sc, tp, P, G, k * kTubeItem, lane);
        }
        cluster_barrier<CL>();  // the peer reads this CTA's G next
        if (tid == 0) sc.work_next2[b] = 0;
    }
}

// Tile pairs at least two tiles apart (I << 16 | J, J >= I + 2), row by row: the
// candidates of the quarter items. Tiles with themselves and with their neighbour are
// listed by index arithmetic.
__device__ void tile_pair_table(const Shared& sm, int nt) {
    const int nfar = nt >= 3 ? (nt - 1) * (nt - 2) / 2 : 0;
    for (int p = threadIdx.x; p < nfar; p += blockDim.x) {
        int I = 0, row = nt - 2, q = p;
        while (q >= row) {
            q -= row;
            ++I;
            --row;
        }
        sm.tpl[p] = ((uint32_t)I << 16) | (uint32_t)(I + 2 + q);
    }
}

}  // namespace

// A CTA pair runs at most kMaxThreadsPair threads per CTA, which leaves 80 registers per
// thread (fewer spills; 2 % faster than 1024 threads with 64 registers, measured); a lone
// CTA per replica keeps 1024 threads, so that two 512-thread CTAs can share an SM.
template <int ELEC, int CL, bool TUBE>
__global__ void __launch_bounds__(CL == 2 ? kMaxThreadsPair : 1024, 1)
k_resident(const TopoDev* __restrict__ topos, const RepDev* __restrict__ reps, StateDev st,
           RunParams P, int nta, int ntp_max, int ncon_max) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Scalars sc;
    const RepDev rep = reps[blockIdx.x / CL];  // this launch's replicas, in any order
    const int r = rep.index;
    const int rank = cta_rank<CL>();
    const TopoDev tp = topos[rep.topo];
    Shared sm = carve(smem_raw, nta, ntp_max, ncon_max);
    const int n = tp.n_atoms, nt = tp.n_tiles;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nta3 = 3 * nta;

    for (int i = tid; i < nta; i += blockDim.x) {
        if (i < n) {
            const float4 x = st.x[rep.atom_off + i];
            sm.xq[i] = make_float4(x.x, x.y, x.z, tp.qs[i]);
            sm.lj[i] = tp.lj[i];
            const float4 v = st.v[rep.atom_off + i];
            sm.v[i] = make_float4(v.x, v.y, v.z, tp.inv_m[i]);
        } else {  // padding: far apart from everything, no charge, no LJ
            sm.xq[i] = make_float4(1.0e5f * (float)(i + 1), 0.f, 0.f, 0.f);
            sm.lj[i] = make_float2(0.f, 0.f);
            sm.v[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    for (int i = tid; i < nta3; i += blockDim.x) {
        sm.Fp[0][i] = 0;
        sm.Fp[1][i] = 0;
        sm.Gp[0][i] = 0;
        sm.Gp[1][i] = 0;
    }
    tile_pair_table(sm, nt);
    if (tid == 0) {
        sc.zm = st.zm[r];
        sc.z = st.z[r];
        sc.T = st.T[r];
        sc.status = st.status[r];
        sc.n_saved = st.n_saved[r];
        sc.flag[0] = 0;
        sc.flag[1] = 0;
        sc.bias_on = 0;
        sc.work_next[0] = 0;
        sc.work_next[1] = 0;
        sc.work_next2[0] = 0;
        sc.work_next2[1] = 0;
        sc.sm = st.sm[r];
        sc.wm = st.wm[r];
    }
    for (int i = tid; i < kMaxTubeK; i += blockDim.x) {
        sc.red_d[0][i] = 0;
        sc.red_d[1][i] = 0;
    }
    long long step = st.step[r];
    __syncthreads();
    all_boxes(sm, n);
    cluster_barrier<CL>();  // every CTA of the cluster is initialised before any remote access
    const int peer = rank ^ 1;
    const float hdt = P.half_dt;
    if (sc.status == 0 && P.n_steps > 0) {
        // the O half step that follows an evaluation uses the noise of the same step index
        evaluate<ELEC, false, CL, TUBE>(sm, sc, tp, P, (int)(step & 1), true, rep.rep_id, step);
        // position of `step` in the save cycle and ring slot of the next frame, kept as
        // counters so that the loop has no 64-bit divisions
        int save_phase = P.save_interval > 0 ? (int)(step % P.save_interval) : -1;
        int slot = P.max_frames > 0 ? (int)(sc.n_saved % P.max_frames) : 0;
        for (long long s = 0; s <= P.n_steps; ++s) {
            // B of the step just evaluated (s > 0), then A of the next one (s < n_steps)
            const bool do_b = s > 0, do_a = s < P.n_steps;
            const int b = (int)(step & 1), nb = b ^ 1;
            const bool bias = sc.bias_on;
            const bool save = do_b && save_phase == 0;
            const float kb = -(float)sc.factor * 4.0f * P.inv_r0sq;  // F_bias = kb G
            for (int base = 0; base < nta; base += blockDim.x) {
                const int i = base + tid;
                const bool valid = i < n;
                float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
                if (valid) {
                    AtomSums a;
                    load_sums<CL>(sm, b, peer, i, bias, a);
                    float4 v = sm.v[i];
                    const float im = v.w;
                    float fx = fix2f(a.f[0]), fy = fix2f(a.f[1]), fz = fix2f(a.f[2]);
                    if (bias) {
                        const float bx = kb * fix2f(a.g[0]), by = kb * fix2f(a.g[1]),
                                    bz = kb * fix2f(a.g[2]);
                        if (do_b) sm.xi[i].w = (bx * bx + by * by + bz * bz) * im;
                        fx += bx;
                        fy += by;
                        fz += bz;
                    }
                    x = sm.xq[i];
                    if (do_b) {  // B: closes the evaluated step
                        v.x = fmaf(hdt * im, fx, v.x);
                        v.y = fmaf(hdt * im, fy, v.y);
                        v.z = fmaf(hdt * im, fz, v.z);
                        if (save && rank == 0) {
                            float* fr = st.frames + 3 * (rep.frame_off + (long long)slot * n + i);
                            fr[0] = x.x;
                            fr[1] = x.y;
                            fr[2] = x.z;
                        }
                    }
                    if (do_a) {  // B A O A of the next step
                        v.x = fmaf(hdt * im, fx, v.x);
                        v.y = fmaf(hdt * im, fy, v.y);
                        v.z = fmaf(hdt * im, fz, v.z);
                        x.x = fmaf(hdt, v.x, x.x);
                        x.y = fmaf(hdt, v.y, x.y);
                        x.z = fmaf(hdt, v.z, x.z);
                        const float4 xi = sm.xi[i];  // drawn during the evaluation
                        v.x = fmaf(P.c1, v.x, xi.x);
                        v.y = fmaf(P.c1, v.y, xi.y);
                        v.z = fmaf(P.c1, v.z, xi.z);
                        x.x = fmaf(hdt, v.x, x.x);
                        x.y = fmaf(hdt, v.y, x.y);
                        x.z = fmaf(hdt, v.z, x.z);
                        if (!(isfinite(x.x) && isfinite(x.y) && isfinite(x.z) && isfinite(v.x) &&
                              isfinite(v.y) && isfinite(v.z)))
                            atomicOr(&sc.status, SCPS_FLAG_NONFINITE);
                        sm.xq[i] = x;
                    }
                    sm.v[i] = v;
                }
                if (do_a) {  // boxes of this warp's tile at the new positions
                    const float4 lo = valid ? x : make_float4(3.0e38f, 3.0e38f, 3.0e38f, 0.f);
                    const float4 hi = valid ? x : make_float4(-3.0e38f, -3.0e38f, -3.0e38f, 0.f);
                    warp_boxes(sm, (base >> 5) + warp, lo, hi, lane);
                }
            }
            if (tid == 0) sc.flag[nb] = 0;
            __syncthreads();
            if (warp == 0 && do_b && bias) {  // atoms in a fixed order, whatever the CTA shape
                float tsum = 0.f;
                for (int i = lane; i < n; i += 32) tsum += sm.xi[i].w;
                tsum = warp_sum_f(tsum);
                if (lane == 0) sc.T += (double)P.dt / P.gamma * (double)tsum;
            }
            if (tid == 0 && do_b) {
                if (save) {
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
            // leave after the last B, or when the new state is non-finite (identical in
            // every CTA of the cluster: same inputs, same arithmetic)
            if (save) slot = slot + 1 == P.max_frames ? 0 : slot + 1;
            if (!do_a || sc.status != 0) break;
            ++step;
            if (save_phase >= 0) save_phase = save_phase + 1 == P.save_interval ? 0 : save_phase + 1;
            const bool save_next = save_phase == 0;
            if (save_next)
                evaluate<ELEC, true, CL, TUBE>(sm, sc, tp, P, nb, true, rep.rep_id, step);
            else
                evaluate<ELEC, false, CL, TUBE>(sm, sc, tp, P, nb, true, rep.rep_id, step);
            if (sc.status != 0) break;  // force out of range: frozen before the update
        }
    }
    __syncthreads();
    // write back the state (rank 0; every CTA holds the same copy)
    if (rank == 0) {
        for (int i = tid; i < n; i += blockDim.x) {
            const float4 x = sm.xq[i];
            st.x[rep.atom_off + i] = make_float4(x.x, x.y, x.z, 0.f);
            const float4 v = sm.v[i];
            st.v[rep.atom_off + i] = make_float4(v.x, v.y, v.z, 0.f);
        }
        if (tid == 0) {
            st.zm[r] = sc.zm;
            st.z[r] = sc.z;
            st.sm[r] = sc.sm;
            st.wm[r] = sc.wm;
            st.T[r] = sc.T;
            st.status[r] = sc.status;
            st.step[r] = step;
            st.n_saved[r] = sc.n_saved;
        }
    }
    cluster_barrier<CL>();  // no CTA leaves while its shared memory may still be read
}

// Energy, forces and z of n_frames configurations (no bias, no state); one cluster of CL
// CTAs per frame. With CL = 2 the work list is split between the two CTAs as in the
// resident kernel and each CTA writes half of the atoms' forces, summing its own and the
// peer's fixed-point partials (the same integers as with one CTA).
template <int ELEC, int CL>
__global__ void __launch_bounds__(1024, 1)
k_eval_frames(const TopoDev* __restrict__ topo_ptr, RunParams P, const float* __restrict__ X,
              double* __restrict__ U, float* __restrict__ F, double* __restrict__ Z, int nta,
              int ntp_max, int ncon_max) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Scalars sc;
    const TopoDev tp = *topo_ptr;
    Shared sm = carve(smem_raw, nta, ntp_max, ncon_max);
    const int n = tp.n_atoms, nt = tp.n_tiles;
    const long long f = blockIdx.x / CL;
    const int rank = cta_rank<CL>();
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
    for (int i = threadIdx.x; i < 3 * nta; i += blockDim.x) {
        sm.Fp[0][i] = 0;
        sm.Gp[0][i] = 0;
    }
    tile_pair_table(sm, nt);
    if (threadIdx.x == 0) {
        sc.zm = 0.0;
        sc.z = 0.0;
        sc.status = 0;
        sc.flag[0] = 0;
        sc.work_next[0] = 0;
    }
    __syncthreads();
    all_boxes(sm, n);
    cluster_barrier<CL>();  // every CTA of the cluster is initialised before any remote access
    evaluate<ELEC, true, CL, false>(sm, sc, tp, P, 0, false, 0u, -1);
    if (F) {  // evaluate ends with a cluster barrier: every partial is complete
        float* ff_out = F + f * n * 3;
        const long long* Fo = rank_ptr<CL>(sm.Fp[0], rank ^ 1);
        for (int i = threadIdx.x + rank * blockDim.x; i < n; i += CL * blockDim.x) {
            long long fx = sm.Fp[0][i], fy = sm.Fp[0][nta + i], fz = sm.Fp[0][2 * nta + i];
            if (CL == 2) {
                fx += Fo[i];
                fy += Fo[nta + i];
                fz += Fo[2 * nta + i];
            }
            ff_out[3 * i] = fix2f(fx);
            ff_out[3 * i + 1] = fix2f(fy);
            ff_out[3 * i + 2] = fix2f(fz);
        }
    }
    if (threadIdx.x == 0 && rank == 0) {
        U[f] = sc.epot;
        if (Z) Z[f] = sc.z;
    }
    cluster_barrier<CL>();  // no CTA leaves while its shared memory may still be read
}

// Shared-memory bytes of the resident kernel for tiles of nta atoms.
size_t resident_smem_bytes(int nta, int ntp_max, int ncon_max) {
    const int nt = nta / kTile;
    const size_t ntp4 = (size_t)((ntp_max + 3) & ~3);
    (void)ncon_max;  // contacts live in the topology (global memory)
    return sizeof(float4) * nta * 3 + sizeof(float4) * 6 * nt + sizeof(long long) * 12 * nta +
           sizeof(float2) * nta + sizeof(uint32_t) * ntp4;
}

// Dynamic shared memory a resident or frame-evaluation CTA may request on the current
// device: the opt-in per-block limit less the largest static shared block of those kernels.
// 0 when the device cannot be queried (nothing then fits).
size_t resident_smem_limit() {
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return 0;
    size_t stat = 0;
    const void* kernels[] = {(const void*)k_resident<ELEC_DDIEL, 1, false>,
                             (const void*)k_resident<ELEC_DDIEL, 2, true>,
                             (const void*)k_eval_frames<ELEC_DDIEL, 1>,
                             (const void*)k_eval_frames<ELEC_DDIEL, 2>};
    for (const void* k : kernels) {
        cudaFuncAttributes a;
        if (cudaFuncGetAttributes(&a, k) != cudaSuccess) return 0;
        stat = std::max(stat, a.sharedSizeBytes);
    }
    return (size_t)optin > stat ? (size_t)optin - stat : 0;
}

template <int ELEC, int CL, bool TUBE>
static cudaError_t launch_resident_t(const TopoDev* topos, const RepDev* reps, const StateDev& st,
                                     const RunParams& P, int nta, int ntp_max, int ncon_max,
                                     int threads, cudaStream_t stream) {
    const size_t smem = resident_smem_bytes(nta, ntp_max, ncon_max);
    auto kern = k_resident<ELEC, CL, TUBE>;
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
    if (P.bias == 5) {  // contact-map tube bias: its own instantiation
        switch (elec) {
            case ELEC_DDIEL: return launch_resident_t<ELEC_DDIEL, CL, true>(topos, reps, st, P, nta, ntp_max, ncon_max, threads, stream);
            case ELEC_RF: return launch_resident_t<ELEC_RF, CL, true>(topos, reps, st, P, nta, ntp_max, ncon_max, threads, stream);
            case ELEC_PLAIN: return launch_resident_t<ELEC_PLAIN, CL, true>(topos, reps, st, P, nta, ntp_max, ncon_max, threads, stream);
            default: return launch_resident_t<ELEC_NONE, CL, true>(topos, reps, st, P, nta, ntp_max, ncon_max, threads, stream);
        }
    }
    switch (elec) {
        case ELEC_DDIEL: return launch_resident_t<ELEC_DDIEL, CL, false>(topos, reps, st, P, nta, ntp_max, ncon_max, threads, stream);
        case ELEC_RF: return launch_resident_t<ELEC_RF, CL, false>(topos, reps, st, P, nta, ntp_max, ncon_max, threads, stream);
        case ELEC_PLAIN: return launch_resident_t<ELEC_PLAIN, CL, false>(topos, reps, st, P, nta, ntp_max, ncon_max, threads, stream);
        default: return launch_resident_t<ELEC_NONE, CL, false>(topos, reps, st, P, nta, ntp_max, ncon_max, threads, stream);
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
                                 int ntp_max, int ncon_max, int threads, int cl,
                                 cudaStream_t stream) {
    const size_t smem = resident_smem_bytes(nta, ntp_max, ncon_max);
    auto kern = cl == 2 ? k_eval_frames<ELEC, 2> : k_eval_frames<ELEC, 1>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(n_frames * cl));
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, kern, topo, P, X, U, F, Z, nta, ntp_max, ncon_max);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_eval(int elec, const TopoDev* topo, const RunParams& P, const float* X,
                        double* U, float* F, double* Z, long long n_frames, int nta, int ntp_max,
                        int ncon_max, int threads, int cl, cudaStream_t stream) {
    switch (elec) {
        case ELEC_DDIEL: return launch_eval_t<ELEC_DDIEL>(topo, P, X, U, F, Z, n_frames, nta, ntp_max, ncon_max, threads, cl, stream);
        case ELEC_RF: return launch_eval_t<ELEC_RF>(topo, P, X, U, F, Z, n_frames, nta, ntp_max, ncon_max, threads, cl, stream);
        case ELEC_PLAIN: return launch_eval_t<ELEC_PLAIN>(topo, P, X, U, F, Z, n_frames, nta, ntp_max, ncon_max, threads, cl, stream);
        default: return launch_eval_t<ELEC_NONE>(topo, P, X, U, F, Z, n_frames, nta, ntp_max, ncon_max, threads, cl, stream);
    }
}

}  // namespace scps
