// Device-side building blocks of the rMD engine: counter-based noise,
// float-float arithmetic, fixed-point force accumulation, the contact-map
// entry of Eq. (Cij) and the pair potential.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace scps {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32
// multiplications with the Weyl key schedule. Counter words: (atom, replica,
// step, stream); key: the 64-bit seed.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Box-Muller on one Philox block: u1 = (a + 1) 2^-32 in (0, 1], u2 = b 2^-32.
__device__ __forceinline__ float4 normals4_f32(uint4 r) {
    const float s32 = 2.3283064365386963e-10f;  // 2^-32
    float4 n;
    float rad = sqrtf(-2.0f * logf(fmaf((float)r.x, s32, s32)));
    float sn, cs;
    sincospif(2.0f * ((float)r.y * s32), &sn, &cs);
    n.x = rad * cs;
    n.y = rad * sn;
    rad = sqrtf(-2.0f * logf(fmaf((float)r.z, s32, s32)));
    sincospif(2.0f * ((float)r.w * s32), &sn, &cs);
    n.z = rad * cs;
    n.w = rad * sn;
    return n;
}

__device__ __forceinline__ double2 normals2_f64(uint32_t a, uint32_t b) {
    const double s32 = 2.3283064365386962890625e-10;
    const double rad = sqrt(-2.0 * log(((double)a + 1.0) * s32));
    double sn, cs;
    sincospi(2.0 * ((double)b * s32), &sn, &cs);
    return make_double2(rad * cs, rad * sn);
}

// ---------------------------------------------------------------------------
// Fixed-point accumulation: forces are summed as int64 multiples of 2^-20
// kJ mol^-1 nm^-1. Integer sums do not depend on the order of the atomic
// additions, so results are bit-reproducible whatever the scheduling.
// The float -> fixed conversion uses only ALU operations (the hardware
// float->int64 conversion is a slow path on this GPU): round(a) for
// |a| < 2^22 comes from the bits of a + 1.5 * 2^23.
// ---------------------------------------------------------------------------
constexpr float kFixScale = 1048576.0f;         // 2^20
constexpr float kFixInv = 9.5367431640625e-07f;  // 2^-20
// Non-bonded pair terms: each s (x_j - x_i) is rounded to 2^-13 units (summed in 32-bit
// registers over a few pairs, then moved to the 2^-20 accumulators), each pair energy to
// 2^-18 units (finer: the many small energies near r_c share one sign, so their rounding
// does not average out); larger pair energies take the 64-bit path.
constexpr float kPairScale = 8192.0f;     // 2^13
constexpr float kPairEScale = 262144.0f;  // 2^18
constexpr float kPairEMax = 8000.0f;

__device__ __forceinline__ long long f2fix(float v) {
    const float a = v * 16.0f;  // v * 2^4: the part above 2^-16 of the 2^-20 grid
    if (fabsf(a) < 4194304.0f) {
        const float magic = 12582912.0f;  // 1.5 * 2^23
        const float t = __fadd_rn(a, magic);
        const int hi = __float_as_int(t) - 0x4B400000;
        const float r = __fsub_rn(a, __fsub_rn(t, magic));  // exact remainder, |r| <= 1/2
        const float t2 = __fmaf_rn(r, 65536.0f, magic);
        const int lo = __float_as_int(t2) - 0x4B400000;
        return ((long long)hi << 16) + (long long)lo;
    }
    return __float2ll_rn(v * kFixScale);  // |v| >= 2^18: rare slow path
}

__device__ __forceinline__ float fix2f(long long v) {
    const int hi = (int)(v >> 32);
    const unsigned lo = (unsigned)(v & 0xffffffffull);
    return fmaf((float)hi, 4294967296.0f, (float)lo) * kFixInv;
}

// ---------------------------------------------------------------------------
// float-float ("double-single") arithmetic (Dekker 1971; Knuth TwoSum;
// FMA-based TwoProd). Used for the native-contact terms of z, whose 1e-9
// relative budget is beyond FP32 while FP64 runs at 1/64 of the FP32 rate here.
// ---------------------------------------------------------------------------
struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ ff fast_two_sum(float a, float b) {  // needs |a| >= |b|
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ ff ff_add(ff x, ff y) {
    ff s = two_sum(x.hi, y.hi);
    const ff t = two_sum(x.lo, y.lo);
    s.lo = __fadd_rn(s.lo, t.hi);
    s = fast_two_sum(s.hi, s.lo);
    s.lo = __fadd_rn(s.lo, t.lo);
    return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ ff ff_add_f(ff x, float y) {
    ff s = two_sum(x.hi, y);
    s.lo = __fadd_rn(s.lo, x.lo);
    return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ ff ff_mul(ff x, ff y) {
    const float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    return fast_two_sum(p, e);
}

__device__ __forceinline__ ff ff_sqr(ff x) {
    const float p = __fmul_rn(x.hi, x.hi);
    float e = __fmaf_rn(x.hi, x.hi, -p);
    e = __fmaf_rn(2.0f * x.hi, x.lo, e);
    return fast_two_sum(p, e);
}

__device__ __forceinline__ ff ff_div(ff x, ff y) {
    const float q1 = __fdiv_rn(x.hi, y.hi);
    // r = x - q1 * y, exactly enough: q1*y.hi via TwoProd
    const float p = __fmul_rn(q1, y.hi);
    const float pe = __fmaf_rn(q1, y.hi, -p);
    float r = __fsub_rn(x.hi, p);
    r = __fadd_rn(r, __fsub_rn(__fsub_rn(x.lo, pe), __fmul_rn(q1, y.lo)));
    const float q2 = __fdiv_rn(r, y.hi);
    return fast_two_sum(q1, q2);
}

__device__ __forceinline__ double ff_to_double(ff x) { return (double)x.hi + (double)x.lo; }

// round(x * 2^40) of a float-float x with 0 <= x.hi <= 1 (a native-contact
// term (C - C0)^2): the z sum is accumulated as int64 multiples of 2^-40, so it
// does not depend on the order in which warps add their terms.
__device__ __forceinline__ long long ff2fix40(ff x) {
    const float magic = 12582912.0f;                     // 1.5 * 2^23
    const float a = x.hi * 1048576.0f;                   // x.hi * 2^20, |a| <= 2^20
    const float t = __fadd_rn(a, magic);
    const int q1 = __float_as_int(t) - 0x4B400000;       // round(a)
    const float rem = __fsub_rn(a, __fsub_rn(t, magic)); // exact, |rem| <= 1/2
    const float b = __fmaf_rn(x.lo, 1099511627776.0f, rem * 1048576.0f);  // (rem + lo 2^20) 2^20
    const int q2 = __float_as_int(__fadd_rn(b, magic)) - 0x4B400000;
    return ((long long)q1 << 20) + (long long)q2;
}

__device__ __forceinline__ ff ff_from_double(double d) {
    const float hi = __double2float_rn(d);
    return {hi, __double2float_rn(d - (double)hi)};
}

// Exact float-float difference b - a of two floats.
__device__ __forceinline__ ff ff_diff(float b, float a) { return two_sum(b, -a); }

// Squared distance in float-float from exact coordinate differences.
__device__ __forceinline__ ff ff_r2(ff dx, ff dy, ff dz) {
    ff s = ff_sqr(dx);
    s = ff_add(s, ff_sqr(dy));
    return ff_add(s, ff_sqr(dz));
}

// The same squared distance from the two positions, with fewer renormalisations: each axis
// gives its exact difference (h, l), h^2 as an exact product pair (p, e) and the cross
// term 2 h l (l^2 is below 2^-48 of h^2); the three p are summed error-free and every
// low-order part is added once before the final renormalisation. Relative error ~1e-14.
__device__ __forceinline__ ff ff_dist2(float4 a, float4 b) {
    const ff dx = two_sum(b.x, -a.x), dy = two_sum(b.y, -a.y), dz = two_sum(b.z, -a.z);
    const float px = __fmul_rn(dx.hi, dx.hi), py = __fmul_rn(dy.hi, dy.hi), pz = __fmul_rn(dz.hi, dz.hi);
    const float qx = __fmaf_rn(2.0f * dx.hi, dx.lo, __fmaf_rn(dx.hi, dx.hi, -px));
    const float qy = __fmaf_rn(2.0f * dy.hi, dy.lo, __fmaf_rn(dy.hi, dy.hi, -py));
    const float qz = __fmaf_rn(2.0f * dz.hi, dz.lo, __fmaf_rn(dz.hi, dz.hi, -pz));
    const ff s1 = two_sum(px, py);
    const ff s2 = two_sum(s1.hi, pz);
    const float low = __fadd_rn(__fadd_rn(s1.lo, s2.lo), __fadd_rn(__fadd_rn(qx, qy), qz));
    return fast_two_sum(s2.hi, low);
}

// Contact-map entry of Eq. (Cij) in u = (r/r0)^2, using the exact rewrite
// (1 - u^3)/(1 - u^5) = (1 + u + u^2) / (1 + u + u^2 + u^3 + u^4).
__device__ __forceinline__ ff contact_C_ff(ff u) {
    // Horner: num = 1 + u (1 + u); den = 1 + u (1 + u (1 + u (1 + u)))
    const ff one_u = ff_add_f(u, 1.0f);
    const ff num = ff_add_f(ff_mul(u, one_u), 1.0f);
    ff d = ff_add_f(ff_mul(u, one_u), 1.0f);
    d = ff_add_f(ff_mul(u, d), 1.0f);
    d = ff_add_f(ff_mul(u, d), 1.0f);
    return ff_div(num, d);
}

// dC/du in FP32.
__device__ __forceinline__ float contact_dC_du(float u) {
    const float num = fmaf(u, u + 1.0f, 1.0f);
    const float u2 = u * u;
    const float den = num + u2 * u + u2 * u2;
    const float dnum = fmaf(2.0f, u, 1.0f);
    const float dden = dnum + 3.0f * u2 + 4.0f * u2 * u;
    return (dnum * den - num * dden) / (den * den);
}

// ---------------------------------------------------------------------------
// Non-bonded pair term (shifted force). Per-atom operands:
//   xq = (x, y, z, qs), lj = (sigma/2, sqrt(24 eps)).
// qs is the charge scaled so that qs_i qs_j is the Coulomb coefficient the
// electrostatics form needs (see the ELEC_* cases). Returns s with
// F_i = s (x_j - x_i), F_j = -F_i; *e receives the pair energy when ENERGY.
// ---------------------------------------------------------------------------
enum { ELEC_NONE = 0, ELEC_DDIEL = 1, ELEC_RF = 2, ELEC_PLAIN = 3 };

struct PairConst {
    float rc, rc2, inv_rc, inv_rc2, inv_rc3;
    float krf, crf;  // reaction field: k_rf, c_rf
    float s_lim;     // largest |s| whose pair terms the 2^-13 integer sums of one item hold
};

// LJ constants of one pair: sigma^2, 24 eps, and (sigma / r_c)^6 with the
// force term at r_c that the shifted force needs.
struct LJPair {
    float sig2, eps24, c6, a_ljc;
};

__device__ __forceinline__ LJPair lj_pair(float sig, float eps24, const PairConst& pc) {
    LJPair q;
    q.sig2 = sig * sig;
    q.eps24 = eps24;
    const float c2 = q.sig2 * pc.inv_rc2;
    q.c6 = c2 * c2 * c2;
    q.a_ljc = eps24 * q.c6 * fmaf(2.0f, q.c6, -1.0f);  // 24 eps (2 c^12 - c^6) at r_c
    return q;
}

template <int ELEC, bool ENERGY>
__device__ __forceinline__ float pair_s_lj(float r2, const LJPair& q, float qq, const PairConst& pc,
                                           float* e) {
    const float inv_r = rsqrtf(r2);
    const float inv_r2 = inv_r * inv_r;
    const float s2 = q.sig2 * inv_r2;
    const float s6 = s2 * s2 * s2;
    const float a_lj = q.eps24 * s6 * fmaf(2.0f, s6, -1.0f);  // 24 eps (2 s^12 - s^6)
    // -phi'(r)/r (coulomb part) and -phi'(r_c)
    float cr, cc;
    if (ELEC == ELEC_DDIEL) {        // phi = (qq/2) / r^2, qq = 2 f q_i q_j / k_dd
        cr = qq * inv_r2 * inv_r2;
        cc = qq * pc.inv_rc3;
    } else if (ELEC == ELEC_RF) {    // phi = qq (1/r + krf r^2 - crf), qq = f q_i q_j
        cr = qq * fmaf(inv_r2, inv_r, -2.0f * pc.krf);
        cc = qq * fmaf(pc.inv_rc2, 1.0f, -2.0f * pc.krf * pc.rc);
    } else if (ELEC == ELEC_PLAIN) { // phi = qq / r
        cr = qq * inv_r2 * inv_r;
        cc = qq * pc.inv_rc2;
    } else {
        cr = 0.0f;
        cc = 0.0f;
    }
    // s = phi'(r)/r - phi'(rc)/r = -(a_lj inv_r2 + cr) + (a_ljc / rc + cc) inv_r
    const float s = fmaf(fmaf(q.a_ljc, pc.inv_rc, cc), inv_r, -fmaf(a_lj, inv_r2, cr));
    if (ENERGY) {
        // phi_sf(r) = phi(r) - phi(rc) + (r - rc) * (-phi'(rc))
        const float r = r2 * inv_r;
        const float e_lj = q.eps24 * (1.0f / 6.0f) * (s6 * s6 - s6);
        const float e_ljc = q.eps24 * (1.0f / 6.0f) * (q.c6 * q.c6 - q.c6);
        float ec, ecc;
        if (ELEC == ELEC_DDIEL) {
            ec = 0.5f * qq * inv_r2;
            ecc = 0.5f * qq * pc.inv_rc2;
        } else if (ELEC == ELEC_RF) {
            ec = qq * (inv_r + pc.krf * r2 - pc.crf);
            ecc = 0.0f;  // the RF form already vanishes at r_c
        } else if (ELEC == ELEC_PLAIN) {
            ec = qq * inv_r;
            ecc = qq * pc.inv_rc;
        } else {
            ec = 0.0f;
            ecc = 0.0f;
        }
        *e = (e_lj - e_ljc) + (ec - ecc) + (r - pc.rc) * fmaf(q.a_ljc, pc.inv_rc, cc);
    }
    return s;
}

template <int ELEC, bool ENERGY>
__device__ __forceinline__ float pair_s(float r2, float sig, float eps24, float qq,
                                        const PairConst& pc, float* e) {
    return pair_s_lj<ELEC, ENERGY>(r2, lj_pair(sig, eps24, pc), qq, pc, e);
}

}  // namespace scps
