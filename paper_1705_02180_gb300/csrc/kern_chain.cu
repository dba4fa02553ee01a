// Resident rMD step kernel for chain replicas, and the frame evaluator.
//
// One thread-block cluster of CL CTAs (CL = 1 or 2) owns one replica for a
// whole launch of n_steps steps. Positions, velocities and fixed-point force
// partials live in shared memory; the CTAs of a cluster split the force work
// between them (the warps of each CTA pull their items from a counter in their
// own shared memory) and read each other's partials through distributed shared
// memory. Every step evaluates
//   bonded terms + non-bonded pairs from a pair list              -grad U
//   z(X) of Eq. (zrMD) from C_ij of Eq. (Cij) in float-float     collective coordinate
//   ratchet of Eq. (FrMD) in FP64 (z < z_m: z_m = z, no bias)   bias force
//   BAOAB update with Philox4x32-10 noise (Eq. Lang)
// and writes a frame every save_interval steps. Every CTA of a cluster
// integrates all atoms of the replica with the same total force, so their
// copies of the state stay identical without being exchanged.
//
// Pair list. Atoms are grouped in blocks of 8 consecutive chain atoms. For each
// block I the list holds, in ascending order, every atom j of a later block that
// lies within r_list = r_c + skin of some atom of I, in chunks of 8 (the last one
// padded with a far-away sentinel slot). A work item is one block against one
// chunk (64 pairs) on a quarter warp: lane l keeps atom j_l of the chunk and takes
// block atom l ^ t at its pair t, so the i-force accumulators move by one xor exchange
// per pair while the j-force stays in place. Pairs inside a block form 28-pair
// items of their own. The list is rebuilt when a bound on the largest displacement
// since the last build reaches skin/2, or after rebuild_every steps, so no pair
// inside r_c is ever missing.
//
// Summation. Every pair term s (x_j - x_i) is rounded to an integer multiple of
// 2^-13 kJ mol^-1 nm^-1 and summed in integers; bonded and bias terms are rounded
// to 2^-20 units. The shared-memory partials are pairs of 32-bit words (a signed
// integer part and an unsigned 2^-20 fraction part) added with 32-bit atomics, so
// every sum is exact and independent of the order of the additions. Results are
// therefore the same bits whichever warp or CTA takes an item, whatever the list
// skin or rebuild cadence, and across a checkpoint and resume.
#include <cooperative_groups.h>

#include <algorithm>
#include <climits>

#include "scps_internal.h"

namespace cg = cooperative_groups;

namespace scps {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kChunk = 32;    // contacts / bonds / angles per work item (one per lane)

// Shared-memory arrays of one CTA. Atom slots: nta real or padding slots plus 8 sentinel
// slots (a block far from everything) that absorb the padding of list chunks.
struct Shared {
    float4* xq;         // (x, y, z, qs), nta + 8
    float4* v;          // velocities (w: 1/m), nta
    float4* xi;         // noise of the next O half step per atom (sd times Gaussian numbers);
                        // w: the atom's |F_bias|^2 / m of the step just closed. During a list
                        // rebuild it holds the block boxes and chunk counts instead.
    float2* lj;         // (sigma/2, sqrt(24 eps)), nta + 8
    int* FH[2];         // force partials of this CTA by parity of the evaluated step:
    unsigned* FL[2];    //   integer part and 2^-20 fraction part, 3 x (nta + 8) each
    int* GH[2];         // partials of sum_p (C - C0) C'(u) (x_p - x_i) over the native
    unsigned* GL[2];    //   contacts this CTA evaluated (the bias gradient without its
                        //   ratchet factor, which is known only once z is complete)
    int* flag;          // force-range flag of the current evaluation
    struct CacheItem* lc;  // this CTA's pair items when they fit (see CacheItem)
    int nta, na8;       // atom slots; accumulator stride (nta + 8)
    int lc_cap;         // capacity of lc in items
};

// A pair item held in shared memory: descriptor, exclusion mask and the chunk's 8 entries
// (the same data as the global item table, mask table and j entries, without their latency).
struct CacheItem {
    uint32_t desc, pad;
    unsigned long long xm;
    uint16_t j[8];
};

struct Scalars {
    int work_next[2];   // this CTA's work counter, by parity of the evaluated step
    int status;         // replica status (identical in every CTA of a cluster)
    int bias_on;
    int flag[2];        // force-range bits raised during the evaluation of a given parity
    int n_items;        // pair items in this CTA's item table
    int cached;         // 1: the items are held in shared memory (Shared::lc)
    int n_diag;         // blocks whose inner pairs this CTA evaluates
    int build_next;     // block counter of a list build
    unsigned vmax2[2];  // largest |v1|^2 + |v2|^2 of the update, by parity (float bits)
    long long pair_slots;  // pairs one evaluation with the current list takes
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

__device__ __forceinline__ Shared carve(void* base, int nta, int lc_cap) {
    Shared s;
    char* p = (char*)base;
    const int na8 = nta + 8;
    s.nta = nta;
    s.na8 = na8;
    s.xq = (float4*)p; p += sizeof(float4) * na8;
    s.v = (float4*)p; p += sizeof(float4) * nta;
    s.xi = (float4*)p; p += sizeof(float4) * nta;
    for (int b = 0; b < 2; ++b) {
        s.FH[b] = (int*)p; p += sizeof(int) * 3 * na8;
        s.FL[b] = (unsigned*)p; p += sizeof(unsigned) * 3 * na8;
        s.GH[b] = (int*)p; p += sizeof(int) * 3 * na8;
        s.GL[b] = (unsigned*)p; p += sizeof(unsigned) * 3 * na8;
    }
    s.lj = (float2*)p; p += sizeof(float2) * na8;
    s.lc = (CacheItem*)p;
    s.lc_cap = lc_cap;
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

// Adds a 2^-20 fixed-point value to a (integer part, fraction part) accumulator.
__device__ __forceinline__ void red_fix20(int* H, unsigned* L, int k, long long v) {
    atomicAdd(&H[k], (int)(v >> 20));
    atomicAdd(&L[k], (unsigned)(v & 0xfffffll));
}

// Adds an integer number of 2^-13 units (the pair terms).
__device__ __forceinline__ void red_fix13(int* H, unsigned* L, int k, int v) {
    atomicAdd(&H[k], v >> 13);
    atomicAdd(&L[k], ((unsigned)v & 0x1fffu) << 7);
}

// Slow path of a pair term: s13 d (2^-13 units, rounded exactly as on the fast path, so the
// sums are the same integers whichever path a pair takes) to atom i and its negative to atom
// j, in 64-bit; a non-finite term or one above 1e9 kJ/mol/nm raises the force-range flag.
__device__ __forceinline__ void add_pair13(const Shared& sm, int* H, unsigned* L, int i, int j,
                                           float s13, float dx, float dy, float dz) {
    const float tx = s13 * dx, ty = s13 * dy, tz = s13 * dz;
    const float lim = 8.192e12f;  // 1e9 in 2^-13 units
    if (!(fabsf(tx) <= lim && fabsf(ty) <= lim && fabsf(tz) <= lim)) atomicOr(sm.flag, SCPS_FLAG_FORCE_RANGE);
    const long long qx = __float2ll_rn(tx) * 128, qy = __float2ll_rn(ty) * 128,
                    qz = __float2ll_rn(tz) * 128;  // 2^-13 to 2^-20 units
    const int s = sm.na8;
    red_fix20(H, L, i, qx);
    red_fix20(H, L, s + i, qy);
    red_fix20(H, L, 2 * s + i, qz);
    red_fix20(H, L, j, -qx);
    red_fix20(H, L, s + j, -qy);
    red_fix20(H, L, 2 * s + j, -qz);
}

// Bonded terms: integer multiples of 2^-13 kJ mol^-1 nm^-1 (one conversion each); a term
// that is non-finite or beyond 2.6e5 kJ mol^-1 nm^-1 (a bond stretched by more than 1 nm)
// raises the force-range flag, which freezes the replica.
__device__ __forceinline__ void add_term13(const Shared& sm, int* H, unsigned* L, int i, float fx,
                                           float fy, float fz) {
    const int s = sm.na8;
    if (!(fmaxf(fabsf(fx), fmaxf(fabsf(fy), fabsf(fz))) < 2.6e5f) ||
        !(isfinite(fx) && isfinite(fy) && isfinite(fz)))
        atomicOr(sm.flag, SCPS_FLAG_FORCE_RANGE);
    red_fix13(H, L, i, __float2int_rn(fx * kPairScale));
    red_fix13(H, L, s + i, __float2int_rn(fy * kPairScale));
    red_fix13(H, L, 2 * s + i, __float2int_rn(fz * kPairScale));
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

// ---------------------------------------------------------------------------
// Pair items
// ---------------------------------------------------------------------------

// List slab of this replica or frame (see scps_internal.h for the layout).
struct ListDev {
    uint16_t* jl;               // j entries of all blocks
    uint32_t* items;            // this CTA's item table
    unsigned long long* excl;   // exclusion masks of this CTA's items
    int nbs;                    // blocks of the slab layout (nta / 8)
};

__device__ __forceinline__ ListDev list_of(unsigned char* slab, int nta, int rank) {
    ListDev L;
    L.nbs = nta >> 3;
    L.jl = (uint16_t*)slab;
    const long long ib = list_items_bytes(L.nbs);
    L.items = (uint32_t*)(slab + list_jl_bytes(L.nbs) + (long long)rank * ib);
    L.excl = (unsigned long long*)(slab + list_jl_bytes(L.nbs) + 2 * ib) +
             (long long)rank * list_items_cap(L.nbs);
    return L;
}

// The 64 pairs of one item (block I against the chunk whose atom j this lane holds) on
// a quarter warp, fast path: integer pair terms summed in 32-bit registers. Items near
// their block (NEARX) take the excluded pairs from the item's mask xm. Returns false (and
// adds nothing) when some |s| of the quarter warp exceeds pc.s_lim, for which the integer
// sums of the item could overflow; the caller then takes the slow path.
template <int ELEC, bool ENERGY, bool NEARX>
__device__ __forceinline__ bool pair_item_fast(const Shared& sm, int* FH, unsigned* FL,
                                               const TopoDev& tp, const PairConst& pc, int I, int j,
                                               unsigned long long xm, int lane, long long& e18) {
    const int l8 = lane & 7, q = lane >> 3;
    // bit t of xr: the pair this lane takes at iteration t (block atom l8 ^ t) is excluded
    const unsigned xr = NEARX ? (unsigned)(xm >> (8 * l8)) & 0xffu : 0u;
    const float4 xj = sm.xq[j];
    const float2 lj = sm.lj[j];
    const int i0 = 8 * I;
    int fix = 0, fiy = 0, fiz = 0, fjx = 0, fjy = 0, fjz = 0;
    long long ei = 0;
    bool bad = false;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const int i = (i0 | l8) ^ t;  // block atom l8 ^ t
        const float4 xi = sm.xq[i];
        const float2 li = sm.lj[i];
        const float dx = xj.x - xi.x, dy = xj.y - xi.y, dz = xj.z - xi.z;
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        bool ok = r2 < pc.rc2;
        if (NEARX) ok = ok && !((xr >> t) & 1u);
        float e = 0.f;
        float s = pair_s<ELEC, ENERGY>(r2, li.x + lj.x, li.y * lj.y, xi.w * xj.w, pc, &e);
        s = ok ? s : 0.0f;
        bad = bad || !(fabsf(s) <= pc.s_lim);
        if (ENERGY) bad = bad || (ok && !(fabsf(e) < kPairEMax));
        const float s13 = s * kPairScale;
        const int tx = __float2int_rn(s13 * dx), ty = __float2int_rn(s13 * dy),
                  tz = __float2int_rn(s13 * dz);
        fix += tx;
        fiy += ty;
        fiz += tz;
        fjx -= tx;
        fjy -= ty;
        fjz -= tz;
        if (ENERGY) ei += ok ? __float2int_rn(e * kPairEScale) : 0;
        if (t < 7) {  // the sums of block atom l8 ^ t go to the lane that takes it next
            fix = __shfl_xor_sync(kFull, fix, t ^ (t + 1));
            fiy = __shfl_xor_sync(kFull, fiy, t ^ (t + 1));
            fiz = __shfl_xor_sync(kFull, fiz, t ^ (t + 1));
        }
    }
    if ((__ballot_sync(kFull, bad) >> (8 * q)) & 0xffu) return false;
    const int s3 = sm.na8, i = (i0 | l8) ^ 7;  // after the last exchange lane l holds atom l ^ 7
    red_fix13(FH, FL, i, fix);
    red_fix13(FH, FL, s3 + i, fiy);
    red_fix13(FH, FL, 2 * s3 + i, fiz);
    red_fix13(FH, FL, j, fjx);
    red_fix13(FH, FL, s3 + j, fjy);
    red_fix13(FH, FL, 2 * s3 + j, fjz);
    if (ENERGY) e18 += ei;
    return true;
}

// Slow path of an item: every pair term goes to both atoms in 64-bit fixed point (rounded
// per pair as on the fast path) with the range check (a force beyond 1e9 kJ/mol/nm or a
// non-finite one freezes the replica).
template <int ELEC, bool ENERGY>
__device__ __noinline__ void pair_item_slow(const Shared& sm, int* FH, unsigned* FL,
                                            const TopoDev& tp, const PairConst& pc, int I, int j,
                                            int lane, long long& e18) {
    const int l8 = lane & 7;
    const float4 xj = sm.xq[j];
    const float2 lj = sm.lj[j];
    for (int t = 0; t < 8; ++t) {
        const int i = 8 * I + ((l8 + t) & 7);
        const float4 xi = sm.xq[i];
        const float2 li = sm.lj[i];
        const float dx = xj.x - xi.x, dy = xj.y - xi.y, dz = xj.z - xi.z;
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        bool ok = r2 < pc.rc2;
        const int dj = j - i + kExclWindow;
        if (dj >= 0 && dj < 2 * kExclWindow && i < tp.n_atoms) ok = ok && !((tp.excl[i] >> dj) & 1ull);
        if (!ok) continue;
        float e = 0.f;
        const float s = pair_s<ELEC, ENERGY>(r2, li.x + lj.x, li.y * lj.y, xi.w * xj.w, pc, &e);
        add_pair13(sm, FH, FL, i, j, s * kPairScale, dx, dy, dz);
        if (ENERGY) e18 += __float2ll_rn(e * kPairEScale);
    }
}

// One batch of four pair items (one per quarter warp) from this CTA's item table.
template <int ELEC, bool ENERGY>
__device__ __forceinline__ void pair_batch(const Shared& sm, int* FH, unsigned* FL, const TopoDev& tp,
                                           const PairConst& pc, const ListDev& L, int n_items,
                                           bool cached, int batch, int lane, long long& e18) {
    const int it = 4 * batch + (lane >> 3);
    int I = 0, j = sm.nta;  // idle quarter: block 0 against the far sentinel slot (zero terms)
    bool near = false;
    unsigned long long xm = 0ull;
    if (it < n_items) {
        if (cached) {
            const CacheItem& c = sm.lc[it];
            const uint32_t d = c.desc;
            I = (int)(d >> 17);
            near = (d >> 16) & 1u;
            j = (int)c.j[lane & 7];
            xm = c.xm;
        } else {
            const uint32_t d = __ldcg(L.items + it);
            I = (int)(d >> 17);
            near = (d >> 16) & 1u;
            j = (int)__ldcg(L.jl + list_jl_off(L.nbs, I) + 8 * (int)(d & 0xffffu) + (lane & 7));
            if (near) xm = __ldcg(L.excl + it);
        }
    }
    bool done;
    if (__any_sync(kFull, near))
        done = pair_item_fast<ELEC, ENERGY, true>(sm, FH, FL, tp, pc, I, j, xm, lane, e18);
    else
        done = pair_item_fast<ELEC, ENERGY, false>(sm, FH, FL, tp, pc, I, j, xm, lane, e18);
    if (!done) pair_item_slow<ELEC, ENERGY>(sm, FH, FL, tp, pc, I, j, lane, e18);
}

// The 28 pairs inside block I on a quarter warp: at round k = 1..4 lane l takes the pair
// (l, (l + k) & 7) (round 4 on lanes 0..3 only), so every pair comes once; the second
// atom's accumulators rotate one lane per round and return home with one exchange.
template <int ELEC, bool ENERGY>
__device__ __forceinline__ void diag_item(const Shared& sm, int* FH, unsigned* FL, const TopoDev& tp,
                                          const PairConst& pc, int I, int lane, long long& e18) {
    const int l8 = lane & 7, q = lane >> 3;
    const int src = (lane & 24) | ((l8 + 1) & 7);
    const int i = 8 * I + l8;
    const float4 xa = sm.xq[i];
    const float2 la = sm.lj[i];
    const unsigned long long em = i < tp.n_atoms ? tp.excl[i] : 0ull;
    int fax = 0, fay = 0, faz = 0, fbx = 0, fby = 0, fbz = 0;
    long long ei = 0;
    bool bad = false;
#pragma unroll
    for (int k = 1; k <= 4; ++k) {
        const int b = 8 * I + ((l8 + k) & 7);
        const float4 xb = sm.xq[b];
        const float2 lb = sm.lj[b];
        const float dx = xb.x - xa.x, dy = xb.y - xa.y, dz = xb.z - xa.z;
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const bool ok = r2 < pc.rc2 && (k < 4 || l8 < 4) && !((em >> (b - i + kExclWindow)) & 1ull);
        float e = 0.f;
        float s = pair_s<ELEC, ENERGY>(r2, la.x + lb.x, la.y * lb.y, xa.w * xb.w, pc, &e);
        s = ok ? s : 0.0f;
        bad = bad || !(fabsf(s) <= pc.s_lim);
        if (ENERGY) bad = bad || (ok && !(fabsf(e) < kPairEMax));
        const float s13 = s * kPairScale;
        const int tx = __float2int_rn(s13 * dx), ty = __float2int_rn(s13 * dy),
                  tz = __float2int_rn(s13 * dz);
        fax += tx;
        fay += ty;
        faz += tz;
        fbx -= tx;
        fby -= ty;
        fbz -= tz;
        if (ENERGY) ei += ok ? __float2int_rn(e * kPairEScale) : 0;
        if (k < 4) {
            fbx = __shfl_sync(kFull, fbx, src);
            fby = __shfl_sync(kFull, fby, src);
            fbz = __shfl_sync(kFull, fbz, src);
        }
    }
    const int home = (lane & 24) | ((l8 + 4) & 7);
    fbx = __shfl_sync(kFull, fbx, home);
    fby = __shfl_sync(kFull, fby, home);
    fbz = __shfl_sync(kFull, fbz, home);
    const int s3 = sm.na8;
    if (!((__ballot_sync(kFull, bad) >> (8 * q)) & 0xffu)) {
        red_fix13(FH, FL, i, fax + fbx);
        red_fix13(FH, FL, s3 + i, fay + fby);
        red_fix13(FH, FL, 2 * s3 + i, faz + fbz);
        if (ENERGY) e18 += ei;
        return;
    }
    for (int k = 1; k <= 4; ++k) {  // slow path (quarter-uniform)
        const int b = 8 * I + ((l8 + k) & 7);
        const float4 xb = sm.xq[b];
        const float2 lb = sm.lj[b];
        const float dx = xb.x - xa.x, dy = xb.y - xa.y, dz = xb.z - xa.z;
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        if (!(r2 < pc.rc2 && (k < 4 || l8 < 4) && !((em >> (b - i + kExclWindow)) & 1ull))) continue;
        float e = 0.f;
        const float s = pair_s<ELEC, ENERGY>(r2, la.x + lb.x, la.y * lb.y, xa.w * xb.w, pc, &e);
        add_pair13(sm, FH, FL, i, b, s * kPairScale, dx, dy, dz);
        if (ENERGY) e18 += __float2ll_rn(e * kPairEScale);
    }
}

// ---------------------------------------------------------------------------
// Bonded terms, contacts, noise
// ---------------------------------------------------------------------------

template <bool ENERGY>
__device__ __forceinline__ float bond_term(const Shared& sm, int* H, unsigned* L, const TopoDev& tp,
                                           int b) {
    const int2 ij = tp.bond_ij[b];
    const float2 par = tp.bond_par[b];
    const float4 a = sm.xq[ij.x], c = sm.xq[ij.y];
    const float dx = c.x - a.x, dy = c.y - a.y, dz = c.z - a.z;
    const float r = sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
    const float dr = r - par.x;
    const float f = par.y * dr / r;
    add_term13(sm, H, L, ij.x, f * dx, f * dy, f * dz);
    add_term13(sm, H, L, ij.y, -f * dx, -f * dy, -f * dz);
    return ENERGY ? 0.5f * par.y * dr * dr : 0.0f;
}

template <bool ENERGY>
__device__ __forceinline__ float angle_term(const Shared& sm, int* H, unsigned* L, const TopoDev& tp,
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
    add_term13(sm, H, L, ijk.x, fix, fiy, fiz);
    add_term13(sm, H, L, ijk.z, fkx, fky, fkz);
    add_term13(sm, H, L, ijk.y, -(fix + fkx), -(fiy + fky), -(fiz + fkz));
    return ENERGY ? 0.5f * par.y * dth * dth : 0.0f;
}

// Adds h (x_p - x_i) to G_i and its negative to G_p (2^-20 fixed point). |h| <= |C - C0|
// |dC/du| < 1 and h |x_p - x_i| stays far below 2^11, so one conversion to a 32-bit count
// of 2^-20 units rounds exactly as the 64-bit conversion would.
__device__ __forceinline__ void add_grad(const Shared& sm, int* GH, unsigned* GL, int i, int p,
                                         float h, float dx, float dy, float dz) {
    const float h20 = h * 1048576.0f;  // 2^20
    const int gx = __float2int_rn(h20 * dx), gy = __float2int_rn(h20 * dy),
              gz = __float2int_rn(h20 * dz);
    const int s = sm.na8;
    red_fix20(GH, GL, i, (long long)gx);
    red_fix20(GH, GL, s + i, (long long)gy);
    red_fix20(GH, GL, 2 * s + i, (long long)gz);
    red_fix20(GH, GL, p, -(long long)gx);
    red_fix20(GH, GL, s + p, -(long long)gy);
    red_fix20(GH, GL, 2 * s + p, -(long long)gz);
}

// One native contact (i, p): (C - C0)^2 in float-float, returned as a 2^-40
// fixed-point value. h (x_p - x_i) with h = (C - C0) dC/du goes to G_i and its
// negative to G_p, so that grad_i (C - C0)^2 = -4 h (x_p - x_i) / r0^2 is
// -4 G_i / r0^2 summed over the atom's contacts (Eq. zrMD, Eq. Cij).
__device__ __forceinline__ long long contact_term(const Shared& sm, int* GH, unsigned* GL,
                                                  const TopoDev& tp, const RunParams& P, int c) {
    const int2 ij = tp.con_ij[c];
    const float4 a = sm.xq[ij.x], b = sm.xq[ij.y];
    const ff r2 = ff_dist2(a, b);
    const ff u = ff_mul(r2, P.inv_r0sq_ff);
    const ff C = contact_C_ff(u);
    const float2 c0 = tp.con_C0[c];
    const ff d = ff_add(C, ff{-c0.x, -c0.y});
    const float h = (d.hi + d.lo) * contact_dC_du(u.hi);
    add_grad(sm, GH, GL, ij.x, ij.y, h, b.x - a.x, b.y - a.y, b.z - a.z);
    return ff2fix40(ff_sqr(d));
}

// Noise of the O half step of global step `step` for atoms 32 q .. 32 q + 31:
// sqrt((1 - c1^2) kT / m_i) times Gaussian numbers from Philox4x32-10 with
// counter (atom, replica id, step, 0). Drawn during the evaluation that precedes the
// O half step, by warps that then go on to pull work items (the update stays short).
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

// Contact-map tube bias, first pass over two items of kTubeItem native contacts, one per
// half warp (c0: the first contact of this half's item; has: the half has an item): the
// items' shares of sum_p (C_p(X) - <C_p(t'_k)>)^2 for every reference slice k, each
// item's share rounded to fixed point (2^-40) and added to the lanes' running sums dacc
// (exact integer sums: independent of which warp takes which item). Half lanes 0..7
// compute C of their item's contacts; then half lane l takes slices l, l + 16, ... The
// reference maps are stored by item, slice-major inside an item (the eight contacts'
// values of one slice side by side, zero past the last contact), so a lane reads the
// eight values of its slice with two 16-byte loads. Lane l keeps the sums of slices l,
// l + 32, ...: of each pair of 16-slice blocks the half keeps one block's values and
// swaps the other with the opposite half.
__device__ __forceinline__ void tube_pass1(const Shared& sm, const TopoDev& tp, const RunParams& P,
                                           int c0, bool has, int lane, long long* dacc) {
    const int hl = lane & 15;
    const bool h1 = lane & 16;
    const int nq = has ? min(kTubeItem, tp.n_contacts - c0) : 0;
    float C = 0.f;
    if (hl < nq) {
        const int2 ij = tp.con_ij[c0 + hl];
        const float4 a = sm.xq[ij.x], q = sm.xq[ij.y];
        const float dx = q.x - a.x, dy = q.y - a.y, dz = q.z - a.z;
        C = contact_C_f32(fmaf(dx, dx, fmaf(dy, dy, dz * dz)) * P.inv_r0sq);
    }
    const int K = P.tube_k;
    const float4* slab = reinterpret_cast<const float4*>(tp.tube_A) + (size_t)(c0 / kTubeItem) * K * 2;
    float even = 0.f;  // this lane's sum of the even block of the current pair of blocks
#pragma unroll
    for (int blk = 0; blk < kMaxTubeK / 16; ++blk) {
        if (blk * 16 >= K) break;
        const int k = blk * 16 + hl;
        const bool in = has && k < K;
        const float4 lo = in ? __ldg(slab + 2 * k) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 hi = in ? __ldg(slab + 2 * k + 1) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float a[kTubeItem] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
        float acc = 0.f;
#pragma unroll
        for (int q = 0; q < kTubeItem; ++q) {
            const float d = __shfl_sync(kFull, C, (lane & 16) | q) - a[q];
            acc = q < nq ? fmaf(d, d, acc) : acc;
        }
        const bool last = (blk + 1) * 16 >= K;
        if ((blk & 1) == 0 && !last) {
            even = acc;
            continue;
        }
        const float e0 = (blk & 1) ? even : acc, o1 = (blk & 1) ? acc : 0.f;
        const float other = __shfl_xor_sync(kFull, h1 ? e0 : o1, 16);
        dacc[blk >> 1] += __float2ll_rn((h1 ? o1 : e0) * 1099511627776.0f) +  // 2^40
                          __float2ll_rn(other * 1099511627776.0f);
    }
}

// Contact-map tube bias, second pass over two items of kTubeItem contacts, one per
// half warp (c0: the first contact of this half's item; has: the half has an item):
// with gamma_k the weights of the ratchet forces on the slices (dF/dD_k), the force on
// the atoms of contact p is beta_p grad C_p with beta_p = (2/N0) sum_k gamma_k
// (C_p - <C_p(t'_k)>); h = beta_p C'(u) goes to G like the z gradient (F = -2/r0^2 G).
// The dots sum_k gamma_k <C_p(t'_k)> are formed with lane l of a half on slices l,
// l + 16, ... (two 16-byte loads per slice, the eight contacts' values side by side)
// and reduced over the half for the eight contacts at once: three exchange steps
// halve the values each lane holds, one more finishes the sums, so half lane L ends
// with the dot of contact L >> 1. The order of every sum is fixed. Two items per warp
// keep twice the loads in flight per L2 round trip.
__device__ __forceinline__ void tube_pass2(const Shared& sm, const Scalars& sc, const TopoDev& tp,
                                           const RunParams& P, int* GH, unsigned* GL, int c0,
                                           bool has, int lane) {
    const int hl = lane & 15;
    const int nq = has ? min(kTubeItem, tp.n_contacts - c0) : 0;
    // the contact of half lane l (l < nq; clamped elsewhere) is read first, so that its
    // latency overlaps the slice loads
    const int2 ij = has ? tp.con_ij[c0 + min(hl, nq - 1)] : make_int2(0, 0);
    const int K = has ? P.tube_k : 0;
    const float4* slab = reinterpret_cast<const float4*>(tp.tube_A) + (size_t)(c0 / kTubeItem) * K * 2;
    float v[kTubeItem];
#pragma unroll
    for (int q = 0; q < kTubeItem; ++q) v[q] = 0.f;
#pragma unroll
    for (int blk = 0; blk < kMaxTubeK / 16; ++blk) {
        if (blk * 16 >= P.tube_k) break;
        const int k = blk * 16 + hl;
        const bool in = k < K;
        const float g = in ? sc.gam[k] : 0.f;
        const float4 lo = in ? __ldg(slab + 2 * k) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 hi = in ? __ldg(slab + 2 * k + 1) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float a[kTubeItem] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
#pragma unroll
        for (int q = 0; q < kTubeItem; ++q) v[q] = fmaf(g, a[q], v[q]);
    }
    const bool b3 = lane & 8, b2 = lane & 4, b1 = lane & 2;
    float w4[4], w2[2];
#pragma unroll
    for (int q = 0; q < 4; ++q)
        w4[q] = (b3 ? v[q + 4] : v[q]) + __shfl_xor_sync(kFull, b3 ? v[q] : v[q + 4], 8);
#pragma unroll
    for (int q = 0; q < 2; ++q)
        w2[q] = (b2 ? w4[q + 2] : w4[q]) + __shfl_xor_sync(kFull, b2 ? w4[q] : w4[q + 2], 4);
    float w1 = (b1 ? w2[1] : w2[0]) + __shfl_xor_sync(kFull, b1 ? w2[0] : w2[1], 2);
    w1 += __shfl_xor_sync(kFull, w1, 1);
    const float dot = __shfl_sync(kFull, w1, (lane & 16) | ((hl & 7) * 2));
    // every lane stays to the end (all exchanges above are full-warp); lanes >= nq
    // of a half hold a copy of its last contact and add nothing
    const bool live = hl < nq;
    const float4 a = sm.xq[ij.x], q = sm.xq[ij.y];
    const float dx = q.x - a.x, dy = q.y - a.y, dz = q.z - a.z;
    const float u = fmaf(dx, dx, fmaf(dy, dy, dz * dz)) * P.inv_r0sq;
    const float C = contact_C_f32(u);
    const float h = live ? 2.0f * tp.tube_inv_n0 * (C * sc.gam_sum - dot) * contact_dC_du(u) : 0.f;
    if (live) add_grad(sm, GH, GL, ij.x, ij.y, h, dx, dy, dz);
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

// Summed fixed-point partials (this CTA + peer) of one atom: force and bias gradient,
// each in 2^-20 units.
struct AtomSums {
    long long f[3], g[3];
};

// Loads the summed partials of atom i for parity b (the peer's through distributed
// shared memory); all loads are issued before any sum is formed.
template <int CL>
__device__ __forceinline__ void load_sums(const Shared& sm, int b, int peer, int i, bool bias,
                                          AtomSums& a) {
    const int s = sm.na8;
    int fh[3], gh[3];
    unsigned fl[3], gl[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        fh[c] = sm.FH[b][c * s + i];
        fl[c] = sm.FL[b][c * s + i];
        gh[c] = bias ? sm.GH[b][c * s + i] : 0;
        gl[c] = bias ? sm.GL[b][c * s + i] : 0u;
    }
    long long lo[3], glo[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        lo[c] = (long long)fl[c];
        glo[c] = (long long)gl[c];
    }
    if (CL == 2) {
        const int* pFH = rank_ptr<CL>(sm.FH[b], peer);
        const unsigned* pFL = rank_ptr<CL>(sm.FL[b], peer);
        const int* pGH = rank_ptr<CL>(sm.GH[b], peer);
        const unsigned* pGL = rank_ptr<CL>(sm.GL[b], peer);
        int rh[3], qh[3];
        unsigned rl[3], ql[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            rh[c] = pFH[c * s + i];
            rl[c] = pFL[c * s + i];
            qh[c] = bias ? pGH[c * s + i] : 0;
            ql[c] = bias ? pGL[c * s + i] : 0u;
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            fh[c] += rh[c];
            gh[c] += qh[c];
            lo[c] += (long long)rl[c];
            glo[c] += (long long)ql[c];
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        a.f[c] = ((long long)fh[c] << 20) + lo[c];
        a.g[c] = ((long long)gh[c] << 20) + glo[c];
    }
}

// ---------------------------------------------------------------------------
// Pair list build
// ---------------------------------------------------------------------------

// Builds the pair list of the positions in shared memory: the block boxes, then for the
// blocks I with I % CL == rank (one warp per block) the ascending list of atoms j of
// later blocks within sqrt(rlist2) of some atom of I, then (after a cluster barrier, so
// that both CTAs' counts and entries are complete) this CTA's item table. Items are
// numbered over all blocks, chunks near a block (first j within the exclusion window of
// the block) first; item k goes to CTA k % CL. Called by every thread of every CTA of
// the cluster; returns after a cluster barrier (the peer has finished reading this
// CTA's counts, which share the xi array's space).
template <int CL>
__device__ void build_list(const Shared& sm, Scalars& sc, const TopoDev& tp, float rlist2,
                           const ListDev& L) {
    const int n = tp.n_atoms, nb = (n + 7) >> 3;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int rank = cta_rank<CL>();
    // scratch in the xi array: boxes (2 nb float4), chunk counts, near-chunk counts
    // and the two prefix arrays (nb ints each)
    float4* blo = sm.xi;
    float4* bhi = sm.xi + nb;
    int* cnt = (int*)(sm.xi + 2 * nb);
    int* cntn = cnt + nb;
    int* pren = cntn + nb;
    int* pref = pren + nb;
    __syncthreads();  // warp 0 may still be summing the bias terms held in the xi array
    if (tid == 0) sc.build_next = 0;
    for (int I = tid; I < nb; I += blockDim.x) {
        float4 lo = make_float4(3.0e38f, 3.0e38f, 3.0e38f, 0.f);
        float4 hi = make_float4(-3.0e38f, -3.0e38f, -3.0e38f, 0.f);
        for (int a = 8 * I; a < min(8 * I + 8, n); ++a) {
            const float4 x = sm.xq[a];
            lo.x = fminf(lo.x, x.x);
            lo.y = fminf(lo.y, x.y);
            lo.z = fminf(lo.z, x.z);
            hi.x = fmaxf(hi.x, x.x);
            hi.y = fmaxf(hi.y, x.y);
            hi.z = fmaxf(hi.z, x.z);
        }
        blo[I] = lo;
        bhi[I] = hi;
    }
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    for (;;) {  // this CTA's blocks, one warp each, pulled in order (early blocks have most work)
        int m = 0;
        if (lane == 0) m = atomicAdd(&sc.build_next, 1);
        const int I = __shfl_sync(kFull, m, 0) * CL + rank;
        if (I >= nb) break;
        const float4 bl = blo[I], bh = bhi[I];
        const int i0 = 8 * I, ia = min(8, n - i0);
        uint16_t* out = L.jl + list_jl_off(L.nbs, I);
        int count = 0, n_near = 0;
        for (int J0 = I + 1; J0 < nb; J0 += 32) {
            const int J = J0 + lane;
            const bool cand = J < nb && box_gap2(bl, bh, blo[J], bhi[J]) < rlist2;
            unsigned cm = __ballot_sync(kFull, cand);
            while (cm) {  // four candidate blocks at a time: lane (c, s) tests atom 8 J_c + s
                int Jc = -1;
                const int c = lane >> 3;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    if (cm) {
                        const int Jk = J0 + __ffs(cm) - 1;
                        cm &= cm - 1;
                        if (k == c) Jc = Jk;
                    }
                }
                const int j = Jc >= 0 ? 8 * Jc + (lane & 7) : n;
                bool hit = false;  // within sqrt(rlist2) of some atom of the block
                if (j < n) {
                    const float4 xj = sm.xq[j];
                    float dmin = 3.0e38f;
                    for (int a = 0; a < ia; ++a) {
                        const float4 xa = sm.xq[i0 + a];
                        const float dx = xj.x - xa.x, dy = xj.y - xa.y, dz = xj.z - xa.z;
                        dmin = fminf(dmin, fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
                    }
                    hit = dmin < rlist2;
                }
                const unsigned hm = __ballot_sync(kFull, hit);
                if (hit) out[count + __popc(hm & lt)] = (uint16_t)j;
                const unsigned nm = __ballot_sync(kFull, hit && j < i0 + 8 + 31);
                count += __popc(hm);
                n_near += __popc(nm);
            }
        }
        const int padded = (count + 7) & ~7;
        if (lane < padded - count) out[count + lane] = (uint16_t)sm.nta;
        if (lane == 0) {
            cnt[I] = padded >> 3;
            cntn[I] = (n_near + 7) >> 3;  // chunks whose first entry is near the block
        }
    }
    __threadfence();  // entries are read back with L2 loads (also by the peer CTA)
    cluster_barrier<CL>();  // every block's entries and counts are complete
    if (warp == 0) {  // prefix sums over blocks: near chunks, then the remaining ones
        int runn = 0, runf = 0;
        for (int I0 = 0; I0 < nb; I0 += 32) {
            const int I = I0 + lane;
            int cn = 0, cf = 0;
            if (I < nb) {
                const int owner = I % CL;
                const int ct = *rank_ptr<CL>(&cnt[I], owner);
                cn = *rank_ptr<CL>(&cntn[I], owner);
                cf = ct - cn;
            }
            int sn = cn, sf = cf;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int yn = __shfl_up_sync(kFull, sn, o), yf = __shfl_up_sync(kFull, sf, o);
                if (lane >= o) {
                    sn += yn;
                    sf += yf;
                }
            }
            if (I < nb) {
                pren[I] = runn + sn - cn;
                pref[I] = runf + sf - cf;
            }
            runn += __shfl_sync(kFull, sn, 31);
            runf += __shfl_sync(kFull, sf, 31);
        }
        const int total = runn + runf;
        if (lane == 0) {
            sc.n_items = (total - rank + CL - 1) / CL;
            sc.cached = sc.n_items <= sm.lc_cap ? 1 : 0;
            sc.n_diag = (nb - rank + CL - 1) / CL;
            sc.work_next[0] = 0;
            sc.work_next[1] = 0;
            sc.pair_slots = 64ll * total + 28ll * nb;  // pairs evaluated per step with this list
        }
        // the total number of near chunks, for the far items' numbering
        if (lane == 0) pref[nb] = runn;
    }
    __syncthreads();
    const int tot_near = pref[nb];
    const bool cached = sc.cached;
    for (int I = warp; I < nb; I += nw) {
        const int owner = I % CL;
        const int ct = *rank_ptr<CL>(&cnt[I], owner), cn = *rank_ptr<CL>(&cntn[I], owner);
        for (int c = lane; c < ct; c += 32) {
            const int k = c < cn ? pren[I] + c : tot_near + pref[I] + (c - cn);
            if (k % CL == rank) {
                const uint32_t d = ((uint32_t)I << 17) | ((uint32_t)(c < cn) << 16) | (uint32_t)c;
                if (cached) {  // the chunk's 8 entries: one 16-byte load (chunks are 16-aligned)
                    CacheItem& ci = sm.lc[k / CL];
                    ci.desc = d;
                    ci.xm = 0ull;
                    *(uint4*)ci.j = __ldcg((const uint4*)(L.jl + list_jl_off(L.nbs, I) + 8 * c));
                } else {
                    L.items[k / CL] = d;
                }
            }
        }
        __syncwarp();  // (the records above are complete before their masks are written)
        // excluded pairs of the near items, in the order the lanes meet them (byte s, bit t:
        // entry s with block atom s ^ t); four chunks per pass, eight lanes each, the
        // block atoms' exclusion words held by lanes 0..7
        const unsigned long long exa = (lane < 8 && 8 * I + lane < n) ? tp.excl[8 * I + lane] : 0ull;
        const uint16_t* e = L.jl + list_jl_off(L.nbs, I);
        for (int c0 = 0; c0 < cn; c0 += 4) {
            const int c = c0 + (lane >> 3), sl = lane & 7;
            const int jj = c < cn ? (int)__ldcg(e + 8 * c + sl) : 0;
            unsigned byte = 0u;
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const int a = sl ^ t, i = 8 * I + a;
                const unsigned long long ex = __shfl_sync(kFull, exa, a);
                const int dj = jj - i + kExclWindow;  // entries lie after the block
                if (c < cn && dj < 2 * kExclWindow && ((ex >> dj) & 1ull)) byte |= 1u << t;
            }
            unsigned long long m = (unsigned long long)byte << (8 * sl);
#pragma unroll
            for (int o = 4; o > 0; o >>= 1) m |= __shfl_xor_sync(kFull, m, o);
            if (sl == 0 && c < cn) {
                const int k = pren[I] + c;
                if (k % CL == rank) {
                    if (cached)
                        sm.lc[k / CL].xm = m;
                    else
                        L.excl[k / CL] = m;
                }
            }
        }
    }
    __threadfence();
    cluster_barrier<CL>();  // the peer is done with this CTA's counts; items are visible
}

// ---------------------------------------------------------------------------
// Force evaluation
// ---------------------------------------------------------------------------

// Force evaluation of the configuration in shared memory (pair list current) for
// the evaluated step of parity b. Work items come from the queue of this CTA; its
// share goes to the parity-b partials; the ratchet decision is taken by every CTA
// from the same fixed-point sums. With noise_step >= 0 the CTA also draws the
// Gaussian numbers of that step's O half step for all atoms (each CTA of a cluster
// integrates every atom). On return the CTA is synchronised.
template <int ELEC, bool ENERGY, int CL, bool TUBE>
__device__ void evaluate(Shared& sm, Scalars& sc, const TopoDev& tp, const RunParams& P,
                         const ListDev& L, int b, bool do_ratchet, uint32_t rep_id,
                         long long noise_step) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int nt = tp.n_tiles;
    int* FH = sm.FH[b];
    unsigned* FL = sm.FL[b];
    int* GH = sm.GH[b];
    unsigned* GL = sm.GL[b];
    sm.flag = &sc.flag[b];
    if (noise_step >= 0)
        for (int q = warp; q < nt; q += nw) noise_chunk(sm, tp, P, rep_id, noise_step, q, lane);
    const int rank = cta_rank<CL>();
    // Work list of this CTA: pair batches (four items from its item table each), blocks
    // with themselves (four per batch), then its shares of the contact, bond and angle
    // chunks (global chunk g belongs to CTA g % CL). Under the contact-map tube bias the
    // contact items are first-pass units of two items of kTubeItem contacts (loads from
    // the reference maps in L2), interleaved one to one with the pair batches so that
    // their memory latency overlaps arithmetic.
    const int n_pb = (sc.n_items + 3) >> 2;
    const int n_db = (sc.n_diag + 3) >> 2;
    const bool tube = TUBE && do_ratchet;  // contact-map tube bias: two work phases
    const int ncon = (P.bias == 1 || P.bias == 5) ? tp.n_contacts : 0;  // frames: z too
    const int g_con = tube ? ((ncon + kTubeItem - 1) / kTubeItem + 1) / 2  // two items a unit
                           : (ncon + kChunk - 1) / kChunk;
    const int g_bond = (tp.n_bonds + kChunk - 1) / kChunk;
    const int g_ang = (tp.n_angles + kChunk - 1) / kChunk;
    const int n_con = (g_con - rank + CL - 1) / CL;
    const int n_bond = (g_bond - rank + CL - 1) / CL;
    const int n_ang = (g_ang - rank + CL - 1) / CL;
    const int m_mix = tube ? min(n_pb, n_con) : 0;
    const int e_pair = n_pb + n_con;          // pair batches and contact items end here
    const int e_diag = e_pair + n_db;
    const int e_bond = e_diag + n_bond;
    const int e_all = e_bond + n_ang;
    int* counter = &sc.work_next[b];
    long long e18 = 0, e20 = 0, zacc = 0;  // fixed point: sums independent of the work order
    long long dacc[TUBE ? kMaxTubeK / 32 : 1];  // first-pass slice sums of this lane
#pragma unroll
    for (int q = 0; q < (TUBE ? kMaxTubeK / 32 : 1); ++q) dacc[q] = 0;
    int m_next = 0;  // the next work index is pulled while the current item runs
    if (lane == 0) m_next = atomicAdd(counter, 1);
    for (;;) {
        const int k = __shfl_sync(kFull, m_next, 0);
        if (k >= e_all) break;
        if (lane == 0) m_next = atomicAdd(counter, 1);
        if (k < e_pair) {
            int kp = -1, kc = -1;  // pair batch or contact item
            if (k < 2 * m_mix) {
                if (k & 1) kc = k >> 1; else kp = k >> 1;
            } else {
                const int r = k - 2 * m_mix;
                if (r < n_pb - m_mix) kp = m_mix + r; else kc = m_mix + r - (n_pb - m_mix);
            }
            if (kp >= 0) {
                pair_batch<ELEC, ENERGY>(sm, FH, FL, tp, P.pc, L, sc.n_items, sc.cached, kp, lane, e18);
            } else {
                const int g = kc * CL + rank;
                if (tube) {
                    if constexpr (TUBE) {
                        const int c0 = (2 * g + (lane >> 4)) * kTubeItem;
                        tube_pass1(sm, tp, P, c0, c0 < ncon, lane, dacc);
                    }
                } else {
                    const int c = g * kChunk + lane;
                    if (c < ncon) zacc += contact_term(sm, GH, GL, tp, P, c);
                }
            }
        } else if (k < e_diag) {
            const int d = 4 * (k - e_pair) + (lane >> 3);
            const int I = d < sc.n_diag ? d * CL + rank : (sm.nta >> 3);
            diag_item<ELEC, ENERGY>(sm, FH, FL, tp, P.pc, I, lane, e18);
        } else if (k < e_bond) {
            const int q = ((k - e_diag) * CL + rank) * kChunk + lane;
            if (q < tp.n_bonds) {
                const float eb = bond_term<ENERGY>(sm, FH, FL, tp, q);
                if (ENERGY) e20 += f2fix(eb);
            }
        } else {
            const int q = ((k - e_bond) * CL + rank) * kChunk + lane;
            if (q < tp.n_angles) {
                const float ea = angle_term<ENERGY>(sm, FH, FL, tp, q);
                if (ENERGY) e20 += f2fix(ea);
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
    long long e = 0;
    if (ENERGY) e = warp_sum_ll((e18 << 2) + e20);  // 2^-18 pair energy units to 2^-20
    if (lane == 0) {
        sc.red_z[b][warp] = zacc;
        sc.red_e[b][warp] = e;
    }
    cluster_barrier<CL>();
    // (the partials of the other parity are cleared atom by atom in the update that follows;
    // the slice sums of the tube bias here)
    if (tube)
        for (int i = tid; i < P.tube_k; i += blockDim.x) sc.red_d[b ^ 1][i] = 0;
    // shares of z, energy and flags from every CTA of the cluster (integer sums); all
    // remote loads are issued before any is used
    if (warp == 0) {
        long long zq[CL], eq[CL];
        int fq[CL];
#pragma unroll
        for (int q = 0; q < CL; ++q) {
            zq[q] = lane < nw ? rank_ptr<CL>(&sc.red_z[b][0], q)[lane] : 0;
            eq[q] = (ENERGY && lane < nw) ? rank_ptr<CL>(&sc.red_e[b][0], q)[lane] : 0;
            fq[q] = lane == 0 ? *rank_ptr<CL>(&sc.flag[b], q) : 0;
        }
        long long zt = 0, et = 0;
        int fl = 0;
#pragma unroll
        for (int q = 0; q < CL; ++q) {
            zt += zq[q];
            et += eq[q];
            fl |= fq[q];
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
        int m2 = 0;  // the next item index is pulled while the current item runs
        if (lane == 0) m2 = atomicAdd(counter2, 1);
        for (;;) {  // units of two items of this CTA, one per half warp
            const int u = __shfl_sync(kFull, m2, 0);
            if (2 * u * CL + rank >= n2) break;
            if (lane == 0) m2 = atomicAdd(counter2, 1);
            const int k = (2 * u + (lane >> 4)) * CL + rank;
            tube_pass2(sm, sc, tp, P, GH, GL, k * kTubeItem, k < n2, lane);
        }
        cluster_barrier<CL>();  // the peer reads this CTA's G next
        if (tid == 0) sc.work_next2[b] = 0;
    }
}

// Atom slots: real atoms, padding slots and the 8 sentinel slots far apart from
// everything (no charge, no LJ).
__device__ __forceinline__ float4 far_slot(int i) {
    return make_float4(1.0e5f * (float)(i + 1), 0.f, 0.f, 0.f);
}

}  // namespace

// A CTA pair runs at most kMaxThreadsPair threads per CTA, which leaves 80 registers per
// thread; a lone CTA per replica keeps 1024 threads, so that two 512-thread CTAs can share
// an SM.
template <int ELEC, int CL, bool TUBE>
__global__ void __launch_bounds__(CL == 2 ? kMaxThreadsPair : 1024, 1)
k_resident(const TopoDev* __restrict__ topos, const RepDev* __restrict__ reps, StateDev st,
           RunParams P, int nta, int lc_cap) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Scalars sc;
    const RepDev rep = reps[blockIdx.x / CL];  // this launch's replicas, in any order
    const int r = rep.index;
    const int rank = cta_rank<CL>();
    const TopoDev tp = topos[rep.topo];
    Shared sm = carve(smem_raw, nta, lc_cap);
    const ListDev L = list_of(P.list_base + rep.list_off, nta, rank);
    const int n = tp.n_atoms;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    for (int i = tid; i < sm.na8; i += blockDim.x) {
        if (i < n) {
            const float4 x = st.x[rep.atom_off + i];
            sm.xq[i] = make_float4(x.x, x.y, x.z, tp.qs[i]);
            sm.lj[i] = tp.lj[i];
            const float4 v = st.v[rep.atom_off + i];
            sm.v[i] = make_float4(v.x, v.y, v.z, tp.inv_m[i]);
        } else {
            sm.xq[i] = far_slot(i);
            sm.lj[i] = make_float2(0.f, 0.f);
            if (i < nta) sm.v[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    for (int i = tid; i < 3 * sm.na8; i += blockDim.x) {
        for (int b = 0; b < 2; ++b) {
            sm.FH[b][i] = 0;
            sm.FL[b][i] = 0u;
            sm.GH[b][i] = 0;
            sm.GL[b][i] = 0u;
        }
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
        sc.work_next[0] = 0;
        sc.work_next[1] = 0;
        sc.work_next2[0] = 0;
        sc.work_next2[1] = 0;
        sc.vmax2[0] = 0u;
        sc.vmax2[1] = 0u;
        sc.sm = st.sm[r];
        sc.wm = st.wm[r];
    }
    for (int i = tid; i < kMaxTubeK; i += blockDim.x) {
        sc.red_d[0][i] = 0;
        sc.red_d[1][i] = 0;
    }
    long long step = st.step[r];
    int builds = 0;  // pair-list builds in this launch
    cluster_barrier<CL>();  // every CTA of the cluster is initialised before any remote access
    const int peer = rank ^ 1;
    const float hdt = P.half_dt;
    if (sc.status == 0 && P.n_steps > 0) {
        build_list<CL>(sm, sc, tp, P.rlist2, L);
        // displacement bound since the last build and steps since then (identical in every
        // thread of the cluster: same inputs, same arithmetic)
        float disp = 0.f;
        int since = 0;
        builds = 1;
        // the O half step that follows an evaluation uses the noise of the same step index
        evaluate<ELEC, false, CL, TUBE>(sm, sc, tp, P, L, (int)(step & 1), true, rep.rep_id, step);
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
            float vm2 = 0.f;  // largest |v after B|^2 + |v after O|^2 of this thread's atoms
            for (int base = 0; base < nta; base += blockDim.x) {
                const int i = base + tid;
                if (i < n) {
                    AtomSums a;
                    load_sums<CL>(sm, b, peer, i, bias, a);
                    // the other parity's partials were last read before this evaluation's
                    // cluster barrier (here and in the peer): clear them for the next one
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        sm.FH[nb][c * sm.na8 + i] = 0;
                        sm.FL[nb][c * sm.na8 + i] = 0u;
                        sm.GH[nb][c * sm.na8 + i] = 0;
                        sm.GL[nb][c * sm.na8 + i] = 0u;
                    }
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
                    float4 x = sm.xq[i];
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
                        const float v1 = fmaf(v.x, v.x, fmaf(v.y, v.y, v.z * v.z));
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
                        vm2 = fmaxf(vm2, v1 + fmaf(v.x, v.x, fmaf(v.y, v.y, v.z * v.z)));
                        if (!(isfinite(x.x) && isfinite(x.y) && isfinite(x.z) && isfinite(v.x) &&
                              isfinite(v.y) && isfinite(v.z)))
                            atomicOr(&sc.status, SCPS_FLAG_NONFINITE);
                        sm.xq[i] = x;
                    }
                    sm.v[i] = v;
                }
            }
            if (do_a) {  // largest speed of the step (positive floats order as their bits)
                const unsigned wm = __reduce_max_sync(kFull, __float_as_uint(vm2));
                if (lane == 0) atomicMax(&sc.vmax2[b], wm);
            }
            if (tid == 0) {
                sc.flag[nb] = 0;
                sc.vmax2[nb] = 0u;
            }
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
            // |x_new - x_old| <= dt/2 (|v after B| + |v after O|) <= dt/2 sqrt(2 vmax2) per
            // atom; a pair inside r_c now was inside r_c + 2 disp at the build, so the list
            // stays complete while 2 disp < skin (a 1 % margin covers the FP32 rounding)
            disp += hdt * sqrtf(2.0f * __uint_as_float(sc.vmax2[b]));
            ++since;
            if (disp >= 0.99f * P.skin_half || (P.rebuild_every > 0 && since >= P.rebuild_every)) {
                build_list<CL>(sm, sc, tp, P.rlist2, L);
                disp = 0.f;
                since = 0;
                ++builds;
            }
            const bool save_next = save_phase == 0;
            if (save_next)
                evaluate<ELEC, true, CL, TUBE>(sm, sc, tp, P, L, nb, true, rep.rep_id, step);
            else
                evaluate<ELEC, false, CL, TUBE>(sm, sc, tp, P, L, nb, true, rep.rep_id, step);
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
            if (st.pair_slots && sc.status == 0 && P.n_steps > 0) st.pair_slots[r] = sc.pair_slots;
            if (st.list_builds) st.list_builds[r] = builds;
        }
    }
    cluster_barrier<CL>();  // no CTA leaves while its shared memory may still be read
}

// Energy, forces and z of n_frames configurations (no bias, no state); one cluster of CL
// CTAs per frame, each cluster with its own list slab. With CL = 2 the work is split
// between the two CTAs as in the resident kernel and each CTA writes half of the atoms'
// forces, summing its own and the peer's fixed-point partials (the same integers as with
// one CTA).
template <int ELEC, int CL>
__global__ void __launch_bounds__(1024, 1)
k_eval_frames(const TopoDev* __restrict__ topo_ptr, RunParams P, const float* __restrict__ X,
              double* __restrict__ U, float* __restrict__ F, double* __restrict__ Z, int nta,
              int lc_cap) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Scalars sc;
    const TopoDev tp = *topo_ptr;
    Shared sm = carve(smem_raw, nta, lc_cap);
    const int n = tp.n_atoms;
    const long long f = blockIdx.x / CL;
    const int rank = cta_rank<CL>();
    const ListDev L = list_of(P.list_base + (blockIdx.x / CL) * P.list_slab, nta, rank);
    const float* xf = X + f * n * 3;
    for (int i = threadIdx.x; i < sm.na8; i += blockDim.x) {
        if (i < n) {
            sm.xq[i] = make_float4(xf[3 * i], xf[3 * i + 1], xf[3 * i + 2], tp.qs[i]);
            sm.lj[i] = tp.lj[i];
        } else {
            sm.xq[i] = far_slot(i);
            sm.lj[i] = make_float2(0.f, 0.f);
        }
    }
    for (int i = threadIdx.x; i < 3 * sm.na8; i += blockDim.x) {
        sm.FH[0][i] = 0;
        sm.FL[0][i] = 0u;
        sm.GH[0][i] = 0;
        sm.GL[0][i] = 0u;
    }
    if (threadIdx.x == 0) {
        sc.zm = 0.0;
        sc.z = 0.0;
        sc.status = 0;
        sc.flag[0] = 0;
        sc.work_next[0] = 0;
    }
    cluster_barrier<CL>();  // every CTA of the cluster is initialised before any remote access
    build_list<CL>(sm, sc, tp, P.rlist2, L);
    evaluate<ELEC, true, CL, false>(sm, sc, tp, P, L, 0, false, 0u, -1);
    if (F) {  // evaluate ends with a cluster barrier: every partial is complete
        float* ff_out = F + f * n * 3;
        const int s = sm.na8;
        const int* oH = rank_ptr<CL>(sm.FH[0], rank ^ 1);
        const unsigned* oL = rank_ptr<CL>(sm.FL[0], rank ^ 1);
        for (int i = threadIdx.x + rank * blockDim.x; i < n; i += CL * blockDim.x) {
            float o[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                int h = sm.FH[0][c * s + i];
                long long l = (long long)sm.FL[0][c * s + i];
                if (CL == 2) {
                    h += oH[c * s + i];
                    l += (long long)oL[c * s + i];
                }
                o[c] = fix2f(((long long)h << 20) + l);
            }
            ff_out[3 * i] = o[0];
            ff_out[3 * i + 1] = o[1];
            ff_out[3 * i + 2] = o[2];
        }
    }
    if (threadIdx.x == 0 && rank == 0) {
        U[f] = sc.epot;
        if (Z) Z[f] = sc.z;
    }
    cluster_barrier<CL>();  // no CTA leaves while its shared memory may still be read
}

// Shared-memory bytes of the resident kernels for nta atom slots (plus the 8 sentinel
// slots): positions, velocities, the xi array, LJ parameters and the two parities of force and
// bias-gradient partials (integer and fraction words).
size_t resident_smem_bytes(int nta) {
    const size_t na8 = (size_t)nta + 8;
    return sizeof(float4) * (na8 + 2 * (size_t)nta) + sizeof(float2) * na8 +
           2 * 4 * 3 * sizeof(int) * na8;
}

// Largest static shared block of the resident and frame-evaluation kernels (0 when the
// device cannot be queried).
static size_t resident_static_smem() {
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
    return stat;
}

// Dynamic shared memory a resident or frame-evaluation CTA may request on the current
// device: the opt-in per-block limit less the largest static shared block of those kernels.
// 0 when the device cannot be queried (nothing then fits).
size_t resident_smem_limit() {
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return 0;
    const size_t stat = resident_static_smem();
    return (size_t)optin > stat ? (size_t)optin - stat : 0;
}

constexpr int kMaxCacheItems = 16384;

// Dynamic shared memory of a launch with CTAs of `threads` threads: the resident state plus
// a cache of pair items (CacheItem, 32 B) in what the state leaves free; CTAs of up to 512
// threads keep room for a second CTA on their SM. Sets *lc_cap to the cache's capacity.
static size_t launch_smem(int nta, int threads, int cl, int* lc_cap) {
    const int cl_items_per_slot = cl == 2 ? 2 : 4;
    const size_t base = resident_smem_bytes(nta);
    size_t lim = resident_smem_limit();
    if (threads <= 512) {
        int dev = 0, per_sm = 0, reserved = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
        const size_t stat = resident_static_smem();
        const size_t two = (size_t)per_sm / 2;
        const size_t half = two > (size_t)reserved + stat ? two - (size_t)reserved - stat : 0;
        lim = std::min(lim, half);
    }
    size_t cap = lim > base ? (lim - base) / sizeof(CacheItem) : 0;
    // no more than the lists of compact chains need (about 1.8 x 80 pairs per atom in items
    // of 64, per CTA): shared memory and the L1 cache share the SM's storage, and the L1
    // serves the topology tables; longer tables stay in global memory
    cap = std::min(cap, std::min((size_t)kMaxCacheItems, (size_t)(cl_items_per_slot * nta)));
    *lc_cap = (int)cap;
    return base + cap * sizeof(CacheItem);
}

template <int ELEC, int CL, bool TUBE>
static cudaError_t launch_resident_t(const TopoDev* topos, const RepDev* reps, const StateDev& st,
                                     const RunParams& P, int nta, int threads, cudaStream_t stream) {
    int lc_cap = 0;
    const size_t smem = launch_smem(nta, threads, CL, &lc_cap);
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
    e = cudaLaunchKernelEx(&cfg, kern, topos, reps, st, P, nta, lc_cap);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <int CL>
static cudaError_t launch_resident_cl(int elec, const TopoDev* topos, const RepDev* reps,
                                      const StateDev& st, const RunParams& P, int nta, int threads,
                                      cudaStream_t stream) {
    if (P.bias == 5) {  // contact-map tube bias: its own instantiation
        switch (elec) {
            case ELEC_DDIEL: return launch_resident_t<ELEC_DDIEL, CL, true>(topos, reps, st, P, nta, threads, stream);
            case ELEC_RF: return launch_resident_t<ELEC_RF, CL, true>(topos, reps, st, P, nta, threads, stream);
            case ELEC_PLAIN: return launch_resident_t<ELEC_PLAIN, CL, true>(topos, reps, st, P, nta, threads, stream);
            default: return launch_resident_t<ELEC_NONE, CL, true>(topos, reps, st, P, nta, threads, stream);
        }
    }
    switch (elec) {
        case ELEC_DDIEL: return launch_resident_t<ELEC_DDIEL, CL, false>(topos, reps, st, P, nta, threads, stream);
        case ELEC_RF: return launch_resident_t<ELEC_RF, CL, false>(topos, reps, st, P, nta, threads, stream);
        case ELEC_PLAIN: return launch_resident_t<ELEC_PLAIN, CL, false>(topos, reps, st, P, nta, threads, stream);
        default: return launch_resident_t<ELEC_NONE, CL, false>(topos, reps, st, P, nta, threads, stream);
    }
}

cudaError_t launch_resident(int elec, int cluster, const TopoDev* topos, const RepDev* reps,
                            const StateDev& st, const RunParams& P, int nta, int threads,
                            cudaStream_t stream) {
    if (cluster == 2) return launch_resident_cl<2>(elec, topos, reps, st, P, nta, threads, stream);
    return launch_resident_cl<1>(elec, topos, reps, st, P, nta, threads, stream);
}

template <int ELEC>
static cudaError_t launch_eval_t(const TopoDev* topo, const RunParams& P, const float* X,
                                 double* U, float* F, double* Z, long long n_frames, int nta,
                                 int threads, int cl, cudaStream_t stream) {
    int lc_cap = 0;
    const size_t smem = launch_smem(nta, threads, cl, &lc_cap);
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
    e = cudaLaunchKernelEx(&cfg, kern, topo, P, X, U, F, Z, nta, lc_cap);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_eval(int elec, const TopoDev* topo, const RunParams& P, const float* X,
                        double* U, float* F, double* Z, long long n_frames, int nta, int threads,
                        int cl, cudaStream_t stream) {
    switch (elec) {
        case ELEC_DDIEL: return launch_eval_t<ELEC_DDIEL>(topo, P, X, U, F, Z, n_frames, nta, threads, cl, stream);
        case ELEC_RF: return launch_eval_t<ELEC_RF>(topo, P, X, U, F, Z, n_frames, nta, threads, cl, stream);
        case ELEC_PLAIN: return launch_eval_t<ELEC_PLAIN>(topo, P, X, U, F, Z, n_frames, nta, threads, cl, stream);
        default: return launch_eval_t<ELEC_NONE>(topo, P, X, U, F, Z, n_frames, nta, threads, cl, stream);
    }
}

}  // namespace scps
