// Solvated periodic box: rMD replicas of one chain in LJ + Coulomb solvent
// (reaction field), cubic box, column-sorted slots and atom-level pair lists.
//
// Per step (kernels in stream order):
//   [rebuild, when due]  wrap; sort atoms into ncol x ncol columns in (x, y),
//                        by z inside a column (ties by atom id); cut every
//                        column into tiles of 32 slots (the last one padded);
//                        inside a tile, order by x into two halves of 16 and
//                        each half by y, so that slots 8q..8q+7 form a compact
//                        cluster; cluster boxes; per 8-slot cluster the list
//                        of atoms of later clusters within r_c + skin of one of
//                        its atoms, each with the periodic shift of its cluster
//                        (the cluster takes the minimum image pair by pair where
//                        that shift might not hold until the next rebuild)
//   pairs                one warp per cluster, four chunks of 8 entries at a
//                        time on quarter warps, every pair once; all force
//                        terms summed in fixed point (order-free)
//   chain                one CTA per replica: bonds, angles, z(X) of Eq.
//                        (zrMD), the ratchet of Eq. (FrMD), the bias force
//   integrate            BAOAB half steps with Philox noise keyed by atom id
// A rebuild is due every `rebuild_every` steps, or earlier when an atom has
// moved more than skin/2 since the last one, so every pair inside the cutoff
// is always in the list; once one live replica is due, all live replicas of the
// batch rebuild together. Forces are integer sums of per-pair terms (order-free);
// positions are wrapped into the box at each rebuild, so runs that rebuild at
// other steps agree to rounding.
#include "scps_internal.h"

namespace scps {

namespace {

constexpr unsigned kFullB = 0xffffffffu;
constexpr int kNumKeys = 8192;  // ncol^2 * nz <= kNumKeys
constexpr int kMaxCols = 256;   // ncol <= 16
constexpr int kSortThreads = 1024;

__device__ __forceinline__ float wrapc(float x, float L, float invL) {
    return x - L * floorf(x * invL);
}

__device__ __forceinline__ float min_img(float d, float L, float invL) {
    return d - L * rintf(d * invL);
}

// number of lanes whose (key, lane) is below this lane's
__device__ __forceinline__ int warp_rank(float key, int lane, bool member, unsigned group) {
    int rank = 0;
#pragma unroll 8
    for (int k = 0; k < 32; ++k) {
        const float kk = __shfl_sync(kFullB, key, k);
        const bool in = (group >> k) & 1u;
        rank += (member && in && (kk < key || (kk == key && k < lane))) ? 1 : 0;
    }
    return rank;
}

}  // namespace

// Rebuild decision of replicas [r0, r0 + nr) by one CTA: a replica rebuilds when forced
// (need set), or, when `auto_ok`, as soon as one live replica of the batch is due (its
// rebuild_every steps are up or its largest displacement reaches skin/2). Lists of all live
// replicas are then rebuilt together: one rebuild of the whole batch keeps the GPU full,
// where replicas due at different steps would each rebuild alone. Values are read before
// any is written, so the decision is the same whatever the thread order. Returns 1 to all
// threads when some replica rebuilds.
__device__ int box_decide_batch(const BoxDev& B, const StateDev& st, int r0, int nr, int auto_ok) {
    int due = 0;
    if (auto_ok)
        for (int r = r0 + threadIdx.x; r < r0 + nr; r += blockDim.x) {
            const float d2 = __uint_as_float(B.maxd2[r]);
            due |= st.status[r] == 0 && (B.since[r] >= B.rebuild_every || d2 >= B.skin2_quarter);
        }
    due = __syncthreads_or(due);
    int any = 0;
    for (int r = r0 + threadIdx.x; r < r0 + nr; r += blockDim.x) {
        const int decide = st.status[r] == 0 && (B.need[r] || due);
        B.need[r] = decide;  // the later rebuild kernels run iff set
        if (decide) {
            B.since[r] = 0;
            B.maxd2[r] = 0u;
            B.nbuild[r] += 1;
        }
        any |= decide;
    }
    return __syncthreads_or(any);
}

// Rebuild, step 1a: the decision (one CTA for the batch); the key counts of the replicas
// that rebuild are cleared by k_box_clear_hist.
__global__ void k_box_decide(BoxDev B, StateDev st, int r0, int nr, int auto_ok) {
    box_decide_batch(B, st, r0, nr, auto_ok);
}

// Graph form of step 1a (one CTA for all R replicas): the same decision, and the graph's
// conditional value: 1 when some replica rebuilds, so that the rebuild kernels run at all
// only then.
__global__ void k_box_decide_graph(BoxDev B, StateDev st, int R, cudaGraphConditionalHandle h) {
    const int any = box_decide_batch(B, st, 0, R, 1);
    if (threadIdx.x == 0) {
        cudaGraphSetConditional(h, any ? 1u : 0u);
        if (any) B.nevent[0] += 1;
    }
}

__global__ void k_box_clear_hist(BoxDev B, int r0) {
    const int r = blockIdx.y + r0;
    if (!B.need[r]) return;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < kNumKeys) B.hist[(size_t)r * kNumKeys + k] = 0;
}

// Rebuild, step 1b (slots): wrap into the box, key = (column, z bin), count keys.
__global__ void k_box_key(BoxDev B, int r0) {
    const int r = blockIdx.y + r0;
    if (!B.need[r]) return;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= B.np) return;
    const size_t base = (size_t)r * B.np;
    B.id2[base + s] = -1;
    const int a = B.id[base + s];
    if (a < 0) return;
    float4 p = B.pos[base + s];
    p.x = wrapc(p.x, B.L, B.invL);
    p.y = wrapc(p.y, B.L, B.invL);
    p.z = wrapc(p.z, B.L, B.invL);
    B.pos[base + s] = p;
    const float cs = (float)B.ncol * B.invL, zs = (float)B.nz * B.invL;
    const int qx = min((int)(p.x * cs), B.ncol - 1), qy = min((int)(p.y * cs), B.ncol - 1),
              qz = min((int)(p.z * zs), B.nz - 1);
    const int k = (qx * B.ncol + qy) * B.nz + qz;
    B.key[base + s] = k;
    atomicAdd(&B.hist[(size_t)r * kNumKeys + k], 1);
}

// Rebuild, step 1c (one CTA of 1024 threads per replica): exclusive scan of the
// key counts (they become running cursors); first compact position and first
// tile of every column (each column starts a tile).
__global__ void __launch_bounds__(kSortThreads) k_box_scan(BoxDev B, int r0) {
    __shared__ int wtot[32];
    const int r = blockIdx.x + r0;
    if (!B.need[r]) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    int* hist = B.hist + (size_t)r * kNumKeys;
    int* col_first = B.colinfo + (size_t)r * 2 * (kMaxCols + 1);
    int* col_tile = col_first + kMaxCols + 1;
    constexpr int kPer = kNumKeys / kSortThreads;
    int loc[kPer], sum = 0;
    const int k0 = tid * kPer;
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
        loc[q] = hist[k0 + q];
        sum += loc[q];
    }
    int x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFullB, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wtot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int t = lane < nw ? wtot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(kFullB, t, o);
            if (lane >= o) t += y;
        }
        wtot[lane] = t;
    }
    __syncthreads();
    int run = (warp > 0 ? wtot[warp - 1] : 0) + x - sum;
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
        hist[k0 + q] = run;
        run += loc[q];
    }
    __syncthreads();
    const int ncols = B.ncol * B.ncol;
    for (int c = tid; c <= ncols; c += blockDim.x) col_first[c] = c < ncols ? hist[c * B.nz] : B.n_atoms;
    __syncthreads();
    if (tid == 0) {
        int t = 0;
        for (int c = 0; c < ncols; ++c) {
            col_tile[c] = t;
            t += (col_first[c + 1] - col_first[c] + 31) >> 5;
        }
        col_tile[ncols] = t;  // <= nt by the capacity ceil(n/32) + ncol^2
    }
}

// Rebuild, step 1d (atoms): scatter into the padded column layout. Within a key
// the atomics give an arbitrary order, which step 1e replaces by atom-id order.
__global__ void k_box_scatter(BoxDev B, int r0) {
    const int r = blockIdx.y + r0;
    if (!B.need[r]) return;
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= B.n_atoms) return;
    const size_t base = (size_t)r * B.np;
    const int* col_first = B.colinfo + (size_t)r * 2 * (kMaxCols + 1);
    const int* col_tile = col_first + kMaxCols + 1;
    const int s = B.slot_of[(size_t)r * B.n_atoms + a];
    const int k = B.key[base + s];
    const int p = atomicAdd(&B.hist[(size_t)r * kNumKeys + k], 1);
    const int c = k / B.nz;
    const int dst = col_tile[c] * 32 + (p - col_first[c]);
    B.pos2[base + dst] = B.pos[base + s];
    B.vel2[base + dst] = B.vel[base + s];
    B.id2[base + dst] = a;
}

// Rebuild, step 1e (keys): put each key's slots in atom-id order (a key holds a
// few atoms); hist[k] now ends key k, so key k spans [hist[k - 1], hist[k]).
__global__ void k_box_keyorder(BoxDev B, int r0) {
    const int r = blockIdx.y + r0;
    if (!B.need[r]) return;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= B.ncol * B.ncol * B.nz) return;
    const int* hist = B.hist + (size_t)r * kNumKeys;
    const int lo = k > 0 ? hist[k - 1] : 0, hi = hist[k];
    if (hi - lo < 2) return;
    const int* col_first = B.colinfo + (size_t)r * 2 * (kMaxCols + 1);
    const int* col_tile = col_first + kMaxCols + 1;
    const int c = k / B.nz;
    const size_t off = (size_t)r * B.np + col_tile[c] * 32 - col_first[c];
    int* id2 = B.id2 + off;
    float4* pos2 = B.pos2 + off;
    float4* vel2 = B.vel2 + off;
    for (int q = lo + 1; q < hi; ++q) {  // insertion sort by id
        const int ia = id2[q];
        const float4 pa = pos2[q], va = vel2[q];
        int u = q - 1;
        while (u >= lo && id2[u] > ia) {
            id2[u + 1] = id2[u];
            pos2[u + 1] = pos2[u];
            vel2[u + 1] = vel2[u];
            --u;
        }
        id2[u + 1] = ia;
        pos2[u + 1] = pa;
        vel2[u + 1] = va;
    }
}

// Rebuild, step 1f (one warp per tile): inside each tile, two halves of 16 by x,
// each ordered by y (padding last), so that slots 8q .. 8q+7 form compact
// clusters; final slot arrays, reference positions, LJ parameters, slot_of.
__global__ void k_box_subsort(BoxDev B, const TopoDev* __restrict__ topo, int r0) {
    const int r = blockIdx.y + r0;
    if (!B.need[r]) return;
    const int t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (t >= B.nt) return;
    const int lane = threadIdx.x & 31;
    const size_t base = (size_t)r * B.np;
    const int s0 = t * 32 + lane;
    const int a = B.id2[base + s0];
    const bool valid = a >= 0;
    const float4 p = B.pos2[base + s0];
    const float4 v = B.vel2[base + s0];
    const float kx = valid ? p.x : 3.0e38f, ky = valid ? p.y : 3.0e38f;
    const int rx = warp_rank(kx, lane, true, kFullB);
    const unsigned upper = __ballot_sync(kFullB, rx >= 16);
    const bool hi = rx >= 16;
    const int ry = warp_rank(ky, lane, true, hi ? upper : ~upper);
    const int s = t * 32 + (hi ? 16 : 0) + ry;
    if (valid) {
        B.pos[base + s] = p;
        B.vel[base + s] = v;
        B.id[base + s] = a;
        B.pos_ref[base + s] = p;
        B.par[base + s] = topo->lj[a];
        B.slot_of[(size_t)r * B.n_atoms + a] = s;
    } else {
        const float4 far = make_float4(1.0e5f * (float)(s + 1), 0.f, 0.f, 0.f);
        B.pos[base + s] = far;
        B.vel[base + s] = make_float4(0.f, 0.f, 0.f, 0.f);
        B.id[base + s] = -1;
        B.pos_ref[base + s] = far;
        B.par[base + s] = make_float2(0.f, 0.f);
    }
}

// Rebuild step 2 (one warp per tile): box of each 8-slot cluster, and whether it holds
// chain atoms or only atoms with the LJ parameters of the last atom (a solvent site), whose
// pair constants the pair kernel then computes once.
__global__ void k_box_tiles(BoxDev B, const TopoDev* __restrict__ topo, int r0) {
    const int r = blockIdx.y + r0;
    if (!B.need[r]) return;
    const int t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (t >= B.nt) return;
    const int lane = threadIdx.x & 31;
    const int s = t * 32 + lane;
    const float4 p = B.pos[(size_t)r * B.np + s];
    const int a = B.id[(size_t)r * B.np + s];
    const bool valid = a >= 0;
    const float2 ref = topo->lj[B.n_atoms - 1];
    const float2 par = B.par[(size_t)r * B.np + s];
    const unsigned pure = __ballot_sync(kFullB, !valid || (par.x == ref.x && par.y == ref.y));
    const unsigned chain = __ballot_sync(kFullB, valid && a < B.n_chain);
    float lx = valid ? p.x : 3.0e38f, ly = valid ? p.y : 3.0e38f, lz = valid ? p.z : 3.0e38f;
    float hx = valid ? p.x : -3.0e38f, hy = valid ? p.y : -3.0e38f, hz = valid ? p.z : -3.0e38f;
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
        lx = fminf(lx, __shfl_xor_sync(kFullB, lx, o));
        ly = fminf(ly, __shfl_xor_sync(kFullB, ly, o));
        lz = fminf(lz, __shfl_xor_sync(kFullB, lz, o));
        hx = fmaxf(hx, __shfl_xor_sync(kFullB, hx, o));
        hy = fmaxf(hy, __shfl_xor_sync(kFullB, hy, o));
        hz = fmaxf(hz, __shfl_xor_sync(kFullB, hz, o));
    }
    if ((lane & 7) == 0) {  // the box of the 8-slot cluster of this lane
        const size_t c = (size_t)r * 4 * B.nt + 4 * t + (lane >> 3);
        const unsigned mine = 0xffu << (lane & ~7);
        const bool cpure = (pure & mine) == mine;
        B.clo[c] = make_float4(lx, ly, lz, cpure ? 1.f : 0.f);
        B.chi[c] = make_float4(hx, hy, hz, 0.f);
        B.cflag[c] = ((chain & mine) ? 1 : 0) | (cpure ? 4 : 0);
    }
}

// Rebuild step 3 (one warp per 8-slot i cluster c): the pair list of c. Its own 8 slots
// come first (the pair kernel takes those pairs once, j slot after i slot); then, from the
// clusters after c in slot order whose boxes come within r_list of c's box, the atoms within
// r_list of some atom of c (minimum-image distances), in ascending slot order. Each entry
// carries the periodic shift s (per axis -1, 0 or 1 in units of L) that takes its cluster's
// box centre nearest to c's. Where a coordinate difference of some atom of c and the entry
// under s, plus the skin (the most two atoms can close in before the next rebuild), reaches
// L / 2, s may stop being the minimum image of that pair: c is then flagged for the per-pair
// minimum image.
__global__ void __launch_bounds__(128) k_box_list(BoxDev B, StateDev st, int r0) {
    __shared__ float4 sxi[4][8];
    __shared__ int col_tile[kMaxCols + 1];  // first tile of each column (and the end)
    const int r = blockIdx.y + r0;
    if (!B.need[r]) return;
    const int ncl = 4 * B.nt;
    const int ncols = B.ncol * B.ncol;
    for (int k = threadIdx.x; k <= ncols; k += blockDim.x)
        col_tile[k] = B.colinfo[(size_t)r * 2 * (kMaxCols + 1) + kMaxCols + 1 + k];
    __syncthreads();
    const int w = threadIdx.x >> 5;
    const int c = blockIdx.x * 4 + w;
    if (c >= ncl) return;
    const int lane = threadIdx.x & 31, l8 = lane & 7, q = lane >> 3;
    const size_t base = (size_t)r * B.np;
    const size_t ci = (size_t)r * ncl + c;
    uint32_t* out = B.ent + ci * B.max_ent;
    constexpr uint32_t kNoShift = (1u << 24) | (1u << 26) | (1u << 28);
    const float4 al = B.clo[ci], ah = B.chi[ci];
    const int si = 8 * c + l8;
    const unsigned ivalid = __ballot_sync(kFullB, B.id[base + si] >= 0) & 0xffu;
    if (lane < 8) {
        sxi[w][lane] = B.pos[base + si];
        out[lane] = (uint32_t)si | kNoShift | (al.w != 0.f ? 1u << 30 : 0u);
    }
    __syncwarp();
    int count = 8;
    bool inexact = false;
    const float room = 0.5f * B.L - 2.0f * sqrtf(B.skin2_quarter);  // L/2 - skin
    if (ivalid) {
        const float cx = 0.5f * (al.x + ah.x), cy = 0.5f * (al.y + ah.y), cz = 0.5f * (al.z + ah.z);
        const float hx = 0.5f * (ah.x - al.x), hy = 0.5f * (ah.y - al.y), hz = 0.5f * (ah.z - al.z);
        // candidate columns: an atom within r_list of c lies at most `reach` columns away in x
        // and in y (periodically); columns in ascending order keep the entries ascending
        const float colw = B.L / (float)B.ncol;
        const int reach = (int)ceilf(sqrtf(B.rlist2) / colw);
        int lo = 0, hi = ncols;  // c's column: the last one whose first tile is <= c's tile
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (col_tile[mid] <= (c >> 2)) lo = mid; else hi = mid;
        }
        const int qx = lo / B.ncol, qy = lo % B.ncol;
        for (int col = 0; col < ncols; ++col) {
            const int ix = col / B.ncol;
            int ddx = abs(ix - qx);
            ddx = min(ddx, B.ncol - ddx);
            if (ddx > reach) {  // the whole row of columns is out of reach
                col = ix * B.ncol + B.ncol - 1;
                continue;
            }
            int ddy = abs(col - ix * B.ncol - qy);
            ddy = min(ddy, B.ncol - ddy);
            if (ddy > reach) continue;
            const int cl1 = 4 * col_tile[col + 1];
            for (int j0 = max(c + 1, 4 * col_tile[col]); j0 < cl1; j0 += 32) {
                const int jc = j0 + lane;
                bool hit = false;
                uint32_t code = 0;
                if (jc < cl1) {
                    const float4 bl = B.clo[(size_t)r * ncl + jc], bh = B.chi[(size_t)r * ncl + jc];
                    if (bl.x <= bh.x) {  // the cluster holds atoms
                        const float dx = 0.5f * (bl.x + bh.x) - cx, dy = 0.5f * (bl.y + bh.y) - cy,
                                    dz = 0.5f * (bl.z + bh.z) - cz;
                        const float sx = -rintf(dx * B.invL), sy = -rintf(dy * B.invL),
                                    sz = -rintf(dz * B.invL);
                        const float ex = fabsf(fmaf(sx, B.L, dx)), ey = fabsf(fmaf(sy, B.L, dy)),
                                    ez = fabsf(fmaf(sz, B.L, dz));
                        const float wx = hx + 0.5f * (bh.x - bl.x), wy = hy + 0.5f * (bh.y - bl.y),
                                    wz = hz + 0.5f * (bh.z - bl.z);
                        // lower bound of any periodic-image distance between the two boxes
                        const float gx = fmaxf(0.f, ex - wx), gy = fmaxf(0.f, ey - wy),
                                    gz = fmaxf(0.f, ez - wz);
                        hit = fmaf(gx, gx, fmaf(gy, gy, gz * gz)) < B.rlist2;
                        code = ((uint32_t)(sx + 1.f) << 24) | ((uint32_t)(sy + 1.f) << 26) |
                               ((uint32_t)(sz + 1.f) << 28) | (bl.w != 0.f ? 1u << 30 : 0u);
                    }
                }
                unsigned m = __ballot_sync(kFullB, hit);
                while (m) {  // four hit clusters at a time: lane 8 k + a takes atom a of the k-th
                    const int nh = min(__popc(m), 4);
                    unsigned mm = m;
                    for (int k = 0; k < q; ++k) mm &= mm - 1u;
                    const int src = __ffs(mm) - 1;  // lane of this quarter's hit cluster (-1: none)
                    const uint32_t hcode = __shfl_sync(kFullB, code, src & 31);
                    for (int k = 0; k < nh; ++k) m &= m - 1u;
                    bool keep = false;
                    uint32_t e = 0;
                    if (q < nh) {
                        const int sj = 8 * (j0 + src) + l8;
                        const int idj = B.id[base + sj];
                        const float4 xj = B.pos[base + sj];  // (loaded with the id: one round trip)
                        if (idj >= 0) {
                            // the atom under its cluster's shift, first against c's box
                            const float px = xj.x + (float)((int)((hcode >> 24) & 3u) - 1) * B.L,
                                        py = xj.y + (float)((int)((hcode >> 26) & 3u) - 1) * B.L,
                                        pz = xj.z + (float)((int)((hcode >> 28) & 3u) - 1) * B.L;
                            const float bx = fmaxf(0.f, fabsf(px - cx) - hx),
                                        by = fmaxf(0.f, fabsf(py - cy) - hy),
                                        bz = fmaxf(0.f, fabsf(pz - cz) - hz);
                            if (fmaf(bx, bx, fmaf(by, by, bz * bz)) < B.rlist2) {
                                // empty slots of c sit far away (x beyond 1e5 nm), so all 8
                                // are tested; dm bounds every per-axis separation from c's atoms
                                float d2 = 3.0e38f;
#pragma unroll
                                for (int t = 0; t < 8; ++t) {
                                    const float4 a = sxi[w][t];
                                    const float dx = px - a.x, dy = py - a.y, dz = pz - a.z;
                                    d2 = fminf(d2, fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
                                }
                                const float dm = fmaxf(fabsf(px - cx) + hx,
                                                       fmaxf(fabsf(py - cy) + hy, fabsf(pz - cz) + hz));
                                if (!(dm < 0.5f * B.L)) {  // the shift may not be the minimum image
                                    d2 = 3.0e38f;
                                    for (int t = 0; t < 8; ++t) {
                                        if (!((ivalid >> t) & 1u)) continue;
                                        const float4 a = sxi[w][t];
                                        const float mx = min_img(xj.x - a.x, B.L, B.invL),
                                                    my = min_img(xj.y - a.y, B.L, B.invL),
                                                    mz = min_img(xj.z - a.z, B.L, B.invL);
                                        d2 = fminf(d2, fmaf(mx, mx, fmaf(my, my, mz * mz)));
                                    }
                                }
                                keep = d2 < B.rlist2;
                                inexact = inexact || (keep && !(dm < room));
                                e = (uint32_t)sj | (hcode & 0x7f000000u);
                            }
                        }
                    }
                    const unsigned kb = __ballot_sync(kFullB, keep);
                    if (keep) {
                        const int pos = count + __popc(kb & ((1u << lane) - 1u));
                        if (pos < B.max_ent) out[pos] = e;
                    }
                    count += __popc(kb);
                }
            }
        }
    }
    const int padded = (count + 7) & ~7;
    const int k = count + lane;
    if (k < padded && k < B.max_ent) out[k] = kBoxNoSlot | (1u << 30);  // padding: far, "pure"
    const bool overflow = padded > B.max_ent;
    const bool any_inexact = __any_sync(kFullB, inexact);
    if (lane == 0) {
        B.nent[ci] = overflow ? (B.max_ent & ~7) : padded;
        if (any_inexact) B.cflag[ci] |= 2;
        if (overflow) atomicOr(&st.status[r], SCPS_FLAG_LIST_OVERFLOW);
    }
}

// The 64 pairs of one chunk (8 list entries) with the 8 atoms of the i cluster, on a quarter
// warp: lane l holds entry j_l; at iteration t it takes cluster atom l ^ t, so the i-force
// sums move by one xor exchange per iteration (after the eighth, xor 7, lane l holds atom
// l's again) while the j force stays in the lane. Each pair term s (x_j - x_i) is rounded to
// 2^-13 units and summed in 32-bit registers. FIRST: quarter 0 holds the cluster's own
// slots, whose pairs count once (j slot after i slot). EXCL: exclusion masks (clusters holding chain atoms); MINIMG:
// per-pair minimum image; FAST: every atom has the reference LJ parameters, whose pair
// constants U are computed once. Returns false for the quarters where some |s| exceeds
// pc.s_lim (their 32-bit sums could overflow; the caller redoes those chunks pair by pair).
template <int ELEC, bool ENERGY, bool EXCL, bool MINIMG, bool FAST, bool FIRST>
__device__ __forceinline__ bool box_chunk(const BoxDev& B, const PairConst& pc, const LJPair& U,
                                          const float4* sx, const float2* sp, const int* sid,
                                          const unsigned long long* sem, float4 xj, float2 lj,
                                          int idj, int lane, int& fix, int& fiy, int& fiz,
                                          int& fjx, int& fjy, int& fjz, long long& e18) {
    const int l8 = lane & 7, q = lane >> 3;
    long long ech = 0;
    bool bad = false;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const int ii = l8 ^ t;
        const float4 xi = sx[ii];
        float dx = xj.x - xi.x, dy = xj.y - xi.y, dz = xj.z - xi.z;
        if (MINIMG) {
            dx = min_img(dx, B.L, B.invL);
            dy = min_img(dy, B.L, B.invL);
            dz = min_img(dz, B.L, B.invL);
        }
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        bool ok = r2 < pc.rc2;
        if (FIRST) ok = ok && (q != 0 || l8 > ii);
        if (MINIMG || EXCL) {
            const int idi = sid[ii];
            if (MINIMG) ok = ok && idj >= 0 && idi >= 0;
            if (EXCL) {
                const unsigned dj = (unsigned)(idj - idi + kExclWindow);
                if (dj < 2u * kExclWindow && idj < B.n_chain) ok = ok && !((sem[ii] >> dj) & 1ull);
            }
        }
        float ep = 0.f, s;
        if (FAST) {
            s = pair_s_lj<ELEC, ENERGY>(r2, U, xi.w * xj.w, pc, &ep);
        } else {
            const float2 li = sp[ii];
            s = pair_s<ELEC, ENERGY>(r2, li.x + lj.x, li.y * lj.y, xi.w * xj.w, pc, &ep);
        }
        s = ok ? s : 0.0f;
        bad = bad || !(fabsf(s) <= pc.s_lim);
        if (ENERGY) bad = bad || (ok && !(fabsf(ep) < kPairEMax));
        const float s13 = s * kPairScale;
        const int tx = __float2int_rn(s13 * dx), ty = __float2int_rn(s13 * dy),
                  tz = __float2int_rn(s13 * dz);
        fix += tx;
        fiy += ty;
        fiz += tz;
        fjx -= tx;
        fjy -= ty;
        fjz -= tz;
        if (ENERGY) ech += ok ? __float2int_rn(ep * kPairEScale) : 0;
        const int m = t < 7 ? t ^ (t + 1) : 7;  // to the lane that takes atom l8 ^ t next
        fix = __shfl_xor_sync(kFullB, fix, m);
        fiy = __shfl_xor_sync(kFullB, fiy, m);
        fiz = __shfl_xor_sync(kFullB, fiz, m);
    }
    const bool good = !((__ballot_sync(kFullB, bad) >> (8 * q)) & 0xffu);
    if (ENERGY && good) e18 += ech;
    return good;
}

// Slow path of one chunk (the quarter of a chunk that failed the fast path): every pair
// term, rounded to 2^-13 units as on the fast path, goes to both slots' 64-bit
// accumulators, so the forces are the same integers on either path.
template <int ELEC, bool ENERGY, bool EXCL, bool MINIMG>
__device__ __noinline__ void box_chunk_slow(const BoxDev& B, const PairConst& pc, const float4* sx,
                                            const float2* sp, const int* sid,
                                            const unsigned long long* sem, float4 xj, float2 lj,
                                            int idj, int sj, int si0, bool first, int lane,
                                            unsigned long long* acc, long long& e18) {
    const int l8 = lane & 7, q = lane >> 3;
    for (int t = 0; t < 8; ++t) {
        const int ii = (l8 + t) & 7;
        const float4 xi = sx[ii];
        float dx = xj.x - xi.x, dy = xj.y - xi.y, dz = xj.z - xi.z;
        if (MINIMG) {
            dx = min_img(dx, B.L, B.invL);
            dy = min_img(dy, B.L, B.invL);
            dz = min_img(dz, B.L, B.invL);
        }
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        bool ok = r2 < pc.rc2;
        if (first) ok = ok && (q != 0 || l8 > ii);
        const int idi = sid[ii];
        if (MINIMG) ok = ok && idj >= 0 && idi >= 0;
        if (EXCL) {
            const unsigned dj = (unsigned)(idj - idi + kExclWindow);
            if (dj < 2u * kExclWindow && idj < B.n_chain) ok = ok && !((sem[ii] >> dj) & 1ull);
        }
        if (!ok) continue;
        float ep = 0.f;
        const float2 li = sp[ii];
        const float s = pair_s<ELEC, ENERGY>(r2, li.x + lj.x, li.y * lj.y, xi.w * xj.w, pc, &ep);
        const float s13 = s * kPairScale;
        const long long tx = __float2ll_rn(s13 * dx) * 128, ty = __float2ll_rn(s13 * dy) * 128,
                        tz = __float2ll_rn(s13 * dz) * 128;  // 2^-13 to 2^-20 units
        const int si = si0 + ii;
        const size_t np = (size_t)B.np;
        atomicAdd(&acc[si], (unsigned long long)tx);
        atomicAdd(&acc[np + si], (unsigned long long)ty);
        atomicAdd(&acc[2 * np + si], (unsigned long long)tz);
        atomicAdd(&acc[sj], (unsigned long long)(-tx));
        atomicAdd(&acc[np + sj], (unsigned long long)(-ty));
        atomicAdd(&acc[2 * np + sj], (unsigned long long)(-tz));
        if (ENERGY) e18 += __float2ll_rn(ep * kPairEScale);
    }
}

// Non-bonded forces of one 8-slot i cluster on one warp, each pair once (Newton's third
// law): its list in chunks of 8 entries, four chunks at a time (quarter q takes chunk
// 4 k + q). After a chunk each lane adds its j sums to the entry's slot (three 64-bit
// atomics, in 2^-20 units) and its i sums to 64-bit registers, which go to the cluster's
// slots at the end, summed over the quarters. Entries carry their periodic shift unless
// MINIMG; padding entries sit far away from everything (MINIMG tests ids instead).
template <int ELEC, bool ENERGY, bool EXCL, bool MINIMG>
__device__ __forceinline__ void box_cluster_forces(const BoxDev& B, const TopoDev& tp,
                                                   const RunParams& P, int r, int c, int lane,
                                                   bool ipure, const float4* sx, const float2* sp,
                                                   const int* sid, const unsigned long long* sem) {
    const size_t base = (size_t)r * B.np;
    const size_t ci = (size_t)r * 4 * B.nt + c;
    const uint32_t* lst = B.ent + ci * B.max_ent;
    const int n = B.nent[ci];
    unsigned long long* acc = (unsigned long long*)(B.facc + 3 * base);
    const float2 ref = tp.lj[B.n_atoms - 1];
    const LJPair U = lj_pair(ref.x + ref.x, ref.y * ref.y, P.pc);
    long long ax = 0, ay = 0, az = 0;  // this lane's share of cluster atom (lane & 7), 2^-13
    long long e18 = 0;
    for (int k0 = 0; k0 < n; k0 += 32) {
        const int k = k0 + lane;
        const uint32_t e = k < n ? __ldg(lst + k) : (kBoxNoSlot | (1u << 30));
        const int sj = (int)(e & kBoxNoSlot);
        const bool real = sj != (int)kBoxNoSlot;
        float4 xj = make_float4(1.0e18f, 0.f, 0.f, 0.f);  // beyond any cutoff
        float2 lj = make_float2(0.f, 0.f);
        int idj = -1;
        if (real) {
            xj = B.pos[base + sj];
            if (!MINIMG) {
                xj.x = fmaf((float)((int)((e >> 24) & 3u) - 1), B.L, xj.x);
                xj.y = fmaf((float)((int)((e >> 26) & 3u) - 1), B.L, xj.y);
                xj.z = fmaf((float)((int)((e >> 28) & 3u) - 1), B.L, xj.z);
            }
            if (EXCL || MINIMG) idj = B.id[base + sj];  // ids serve exclusions and the image test
        }
        bool fast = false;
        if constexpr (!EXCL && !MINIMG) fast = __all_sync(kFullB, ipure && ((e >> 30) & 1u));
        if (real && !fast) lj = B.par[base + sj];  // the fast path takes the reference constants
        int fix = 0, fiy = 0, fiz = 0, fjx = 0, fjy = 0, fjz = 0;
        bool good;
        if (k0 == 0) {
            if (fast)
                good = box_chunk<ELEC, ENERGY, false, false, true, true>(
                    B, P.pc, U, sx, sp, sid, sem, xj, lj, idj, lane, fix, fiy, fiz, fjx, fjy, fjz, e18);
            else
                good = box_chunk<ELEC, ENERGY, EXCL, MINIMG, false, true>(
                    B, P.pc, U, sx, sp, sid, sem, xj, lj, idj, lane, fix, fiy, fiz, fjx, fjy, fjz, e18);
        } else {
            if (fast)
                good = box_chunk<ELEC, ENERGY, false, false, true, false>(
                    B, P.pc, U, sx, sp, sid, sem, xj, lj, idj, lane, fix, fiy, fiz, fjx, fjy, fjz, e18);
            else
                good = box_chunk<ELEC, ENERGY, EXCL, MINIMG, false, false>(
                    B, P.pc, U, sx, sp, sid, sem, xj, lj, idj, lane, fix, fiy, fiz, fjx, fjy, fjz, e18);
        }
        if (good) {
            ax += fix;
            ay += fiy;
            az += fiz;
            if (real) {
                atomicAdd(&acc[sj], (unsigned long long)((long long)fjx * 128));
                atomicAdd(&acc[B.np + sj], (unsigned long long)((long long)fjy * 128));
                atomicAdd(&acc[2 * (size_t)B.np + sj], (unsigned long long)((long long)fjz * 128));
            }
        } else {
            if (real && fast) lj = B.par[base + sj];  // the slow path uses the general form
            box_chunk_slow<ELEC, ENERGY, EXCL, MINIMG>(B, P.pc, sx, sp, sid, sem, xj, lj, idj, sj,
                                                      8 * c, k0 == 0, lane, acc, e18);
        }
    }
    // the four quarters' shares of each cluster atom
    ax += __shfl_xor_sync(kFullB, ax, 8);
    ay += __shfl_xor_sync(kFullB, ay, 8);
    az += __shfl_xor_sync(kFullB, az, 8);
    ax += __shfl_xor_sync(kFullB, ax, 16);
    ay += __shfl_xor_sync(kFullB, ay, 16);
    az += __shfl_xor_sync(kFullB, az, 16);
    if (lane < 8 && sid[lane] >= 0) {
        const int si = 8 * c + lane;
        atomicAdd(&acc[si], (unsigned long long)(ax * 128));
        atomicAdd(&acc[B.np + si], (unsigned long long)(ay * 128));
        atomicAdd(&acc[2 * (size_t)B.np + si], (unsigned long long)(az * 128));
    }
    if (ENERGY) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) e18 += __shfl_xor_sync(kFullB, e18, o);
        if (lane == 0 && e18 != 0) atomicAdd((unsigned long long*)&B.epair[r], (unsigned long long)e18);
    }
}

// Non-bonded forces: one warp per 8-slot i cluster, the variant chosen by its flags.
template <int ELEC, bool ENERGY>
__global__ void __launch_bounds__(128, 8) k_box_pairs(BoxDev B, const TopoDev* __restrict__ topo,
                                                   RunParams P, int r0) {
    __shared__ float4 sx[4][8];
    __shared__ float2 sp[4][8];
    __shared__ int sid[4][8];
    __shared__ unsigned long long sem[4][8];
    const int r = blockIdx.y + r0;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = blockIdx.x * 4 + w;
    if (c >= 4 * B.nt) return;
    const TopoDev& tp = *topo;
    if (lane < 8) {
        const size_t sl = (size_t)r * B.np + 8 * c + lane;
        sx[w][lane] = B.pos[sl];
        sp[w][lane] = B.par[sl];
        const int a = B.id[sl];
        sid[w][lane] = a;
        sem[w][lane] = (a >= 0 && a < B.n_chain) ? tp.excl[a] : 0ull;
    }
    __syncwarp();
    const int fl = B.cflag[(size_t)r * 4 * B.nt + c];
    const bool pure = (fl & 4) != 0;
    switch (fl & 3) {
        case 0: box_cluster_forces<ELEC, ENERGY, false, false>(B, tp, P, r, c, lane, pure, sx[w], sp[w], sid[w], sem[w]); break;
        case 1: box_cluster_forces<ELEC, ENERGY, true, false>(B, tp, P, r, c, lane, pure, sx[w], sp[w], sid[w], sem[w]); break;
        default: box_cluster_forces<ELEC, ENERGY, true, true>(B, tp, P, r, c, lane, pure, sx[w], sp[w], sid[w], sem[w]); break;
    }
}

// Total non-bonded force on slot s of replica r (fixed point), which is cleared for the
// next evaluation.
__device__ __forceinline__ float4 take_nb_force(const BoxDev& B, int r, int s) {
    const size_t base = (size_t)r * B.np;
    long long* acc = B.facc + 3 * base;
    float4 f = make_float4(fix2f(acc[s]), fix2f(acc[B.np + s]), fix2f(acc[2 * B.np + s]), 0.f);
    acc[s] = 0;
    acc[B.np + s] = 0;
    acc[2 * B.np + s] = 0;
    return f;
}

// Chain terms of one replica: bonds, angles (minimum image), z and the ratchet,
// the bias force; writes fch (bonded + bias) per chain atom. Also closes the
// rebuild bookkeeping of the step.
template <bool ENERGY>
__global__ void __launch_bounds__(512) k_box_chain(BoxDev B, const TopoDev* __restrict__ topo,
                                                   StateDev st, RunParams P, int r0,
                                                   int do_ratchet, int count_step) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ long long zred[16];
    __shared__ double ered[16];
    __shared__ double s_factor;
    __shared__ int s_bias;
    const int r = blockIdx.x + r0;
    const TopoDev tp = *topo;
    const int nch = B.n_chain, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float4* x = (float4*)smem_raw;                       // nch chain positions
    long long* F = (long long*)(x + nch);                // 3 nch fixed point
    float* hc = (float*)(F + 3 * nch);                   // contacts
    const size_t base = (size_t)r * B.np;
    for (int a = tid; a < nch; a += blockDim.x) x[a] = B.pos[base + B.slot_of[(size_t)r * B.n_atoms + a]];
    for (int i = tid; i < 3 * nch; i += blockDim.x) F[i] = 0;
    __syncthreads();
    const float L = B.L, iL = B.invL;
    double eb = 0.0;
    for (int b = tid; b < tp.n_bonds; b += blockDim.x) {
        const int2 ij = tp.bond_ij[b];
        const float2 par = tp.bond_par[b];
        const float dx = min_img(x[ij.y].x - x[ij.x].x, L, iL), dy = min_img(x[ij.y].y - x[ij.x].y, L, iL),
                    dz = min_img(x[ij.y].z - x[ij.x].z, L, iL);
        const float rr = sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
        const float dr = rr - par.x;
        const float f = par.y * dr / rr;
        const long long qx = f2fix(f * dx), qy = f2fix(f * dy), qz = f2fix(f * dz);
        atomicAdd((unsigned long long*)&F[3 * ij.x], (unsigned long long)qx);
        atomicAdd((unsigned long long*)&F[3 * ij.x + 1], (unsigned long long)qy);
        atomicAdd((unsigned long long*)&F[3 * ij.x + 2], (unsigned long long)qz);
        atomicAdd((unsigned long long*)&F[3 * ij.y], (unsigned long long)(-qx));
        atomicAdd((unsigned long long*)&F[3 * ij.y + 1], (unsigned long long)(-qy));
        atomicAdd((unsigned long long*)&F[3 * ij.y + 2], (unsigned long long)(-qz));
        if (ENERGY) eb += 0.5 * (double)par.y * (double)dr * (double)dr;
    }
    for (int q = tid; q < tp.n_angles; q += blockDim.x) {
        const int4 ijk = tp.ang_ijk[q];
        const float2 par = tp.ang_par[q];
        const float ux = min_img(x[ijk.x].x - x[ijk.y].x, L, iL), uy = min_img(x[ijk.x].y - x[ijk.y].y, L, iL),
                    uz = min_img(x[ijk.x].z - x[ijk.y].z, L, iL);
        const float wx = min_img(x[ijk.z].x - x[ijk.y].x, L, iL), wy = min_img(x[ijk.z].y - x[ijk.y].y, L, iL),
                    wz = min_img(x[ijk.z].z - x[ijk.y].z, L, iL);
        const float cx = uy * wz - uz * wy, cy = uz * wx - ux * wz, cz = ux * wy - uy * wx;
        const float sn = sqrtf(fmaf(cx, cx, fmaf(cy, cy, cz * cz)));
        const float cs = fmaf(ux, wx, fmaf(uy, wy, uz * wz));
        const float ru2 = fmaf(ux, ux, fmaf(uy, uy, uz * uz));
        const float rw2 = fmaf(wx, wx, fmaf(wy, wy, wz * wz));
        const float dth = atan2f(sn, cs) - par.x;
        const float g = -par.y * dth / sn;
        const float au = cs / ru2, aw = cs / rw2;
        const float f1x = g * fmaf(au, ux, -wx), f1y = g * fmaf(au, uy, -wy), f1z = g * fmaf(au, uz, -wz);
        const float f3x = g * fmaf(aw, wx, -ux), f3y = g * fmaf(aw, wy, -uy), f3z = g * fmaf(aw, wz, -uz);
        const long long a1 = f2fix(f1x), a2 = f2fix(f1y), a3 = f2fix(f1z);
        const long long c1 = f2fix(f3x), c2 = f2fix(f3y), c3 = f2fix(f3z);
        atomicAdd((unsigned long long*)&F[3 * ijk.x], (unsigned long long)a1);
        atomicAdd((unsigned long long*)&F[3 * ijk.x + 1], (unsigned long long)a2);
        atomicAdd((unsigned long long*)&F[3 * ijk.x + 2], (unsigned long long)a3);
        atomicAdd((unsigned long long*)&F[3 * ijk.z], (unsigned long long)c1);
        atomicAdd((unsigned long long*)&F[3 * ijk.z + 1], (unsigned long long)c2);
        atomicAdd((unsigned long long*)&F[3 * ijk.z + 2], (unsigned long long)c3);
        atomicAdd((unsigned long long*)&F[3 * ijk.y], (unsigned long long)(-a1 - c1));
        atomicAdd((unsigned long long*)&F[3 * ijk.y + 1], (unsigned long long)(-a2 - c2));
        atomicAdd((unsigned long long*)&F[3 * ijk.y + 2], (unsigned long long)(-a3 - c3));
        if (ENERGY) eb += 0.5 * (double)par.y * (double)dth * (double)dth;
    }
    // z of Eq. (zrMD): (C - C0)^2 in float-float, summed in 2^-40 fixed point
    long long zacc = 0;
    if (P.bias == 1) {
        for (int c = tid; c < tp.n_contacts; c += blockDim.x) {
            const int2 ij = tp.con_ij[c];
            const float4 a = x[ij.x], b = x[ij.y];
            // exact float-float separation, then the minimum-image shift (a multiple of L)
            ff dx = ff_diff(b.x, a.x), dy = ff_diff(b.y, a.y), dz = ff_diff(b.z, a.z);
            dx = ff_add_f(dx, -L * rintf((b.x - a.x) * iL));
            dy = ff_add_f(dy, -L * rintf((b.y - a.y) * iL));
            dz = ff_add_f(dz, -L * rintf((b.z - a.z) * iL));
            const ff u = ff_mul(ff_r2(dx, dy, dz), P.inv_r0sq_ff);
            const ff C = contact_C_ff(u);
            const float2 c0 = tp.con_C0[c];
            const ff d = ff_add(C, ff{-c0.x, -c0.y});
            hc[c] = (d.hi + d.lo) * contact_dC_du(u.hi);
            zacc += ff2fix40(ff_sqr(d));
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        zacc += __shfl_down_sync(kFullB, zacc, o);
        eb += __shfl_down_sync(kFullB, eb, o);
    }
    if (lane == 0) {
        zred[warp] = zacc;
        ered[warp] = eb;
    }
    __syncthreads();
    if (tid == 0) {
        long long zt = 0;
        double et = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            zt += zred[w];
            et += ered[w];
        }
        double factor = 0.0;
        if (P.bias == 1) {
            const double z = (double)zt * 9.094947017729282e-13;  // 2^-40
            st.z[r] = z;
            if (do_ratchet) {  // Eq. (FrMD) with theta(0) = 1
                if (z < st.zm[r])
                    st.zm[r] = z;
                else
                    factor = -P.k_R * (z - st.zm[r]);
            }
        }
        s_factor = factor;
        s_bias = factor != 0.0;
        if (ENERGY) B.eb[r] = et;
        if (B.need[r])
            B.need[r] = 0;  // the rebuild of this step is complete
        else if (count_step)
            B.since[r] += 1;
    }
    __syncthreads();
    const float k = -(float)s_factor * 4.0f * P.inv_r0sq;
    float tb = 0.f;
    for (int a = tid; a < nch; a += blockDim.x) {
        float bx = 0.f, by = 0.f, bz = 0.f;
        if (s_bias) {
            const float4 xa = x[a];
            for (int q = tp.con_off[a]; q < tp.con_off[a + 1]; ++q) {
                const int2 cp = tp.con_nbr[q];
                const float4 xp = x[cp.y];
                const float h = hc[cp.x];
                bx = fmaf(h, min_img(xp.x - xa.x, L, iL), bx);
                by = fmaf(h, min_img(xp.y - xa.y, L, iL), by);
                bz = fmaf(h, min_img(xp.z - xa.z, L, iL), bz);
            }
            bx *= k;
            by *= k;
            bz *= k;
            tb += (bx * bx + by * by + bz * bz) * tp.inv_m[a];
        }
        B.fch[(size_t)r * nch + a] = make_float4(fix2f(F[3 * a]) + bx, fix2f(F[3 * a + 1]) + by,
                                                 fix2f(F[3 * a + 2]) + bz, 0.f);
    }
    // bias functional: fixed order (lane tree, then warps in index order)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tb += __shfl_down_sync(kFullB, tb, o);
    __shared__ float tred[16];
    if (lane == 0) tred[warp] = tb;
    __syncthreads();
    if (tid == 0 && s_bias && count_step) {
        float ts = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) ts += tred[w];
        st.T[r] += (double)P.dt / P.gamma * (double)ts;
    }
}

// BAOAB half steps per slot: B closes the evaluated step, A starts the next one. The largest
// squared displacement since the list build goes to the replica's bound with one atomic per
// warp (every lane reaches the warp reduction; the slots of a warp share their replica).
__global__ void k_box_integrate(BoxDev B, const TopoDev* __restrict__ topo, StateDev st,
                                RunParams P, const uint32_t* __restrict__ rep_ids, long long step,
                                int do_b, int do_a, int step_from_state) {
    const int r = blockIdx.y;
    if (step_from_state) step = st.step[r];  // graph form: the counter the step graph advanced
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const size_t base = (size_t)r * B.np;
    float d2 = 0.f;
    if (s < B.np) {
        float4 f = take_nb_force(B, r, s);  // also clears the j part (frozen replicas too)
        const int a = B.id[base + s];
        if (a >= 0 && st.status[r] == 0) {
            const TopoDev& tp = *topo;
            if (a < B.n_chain) {
                const float4 c = B.fch[(size_t)r * B.n_chain + a];
                f.x += c.x;
                f.y += c.y;
                f.z += c.z;
            }
            const float im = tp.inv_m[a];
            const float hdt = P.half_dt;
            float4 v = B.vel[base + s];
            float4 x = B.pos[base + s];
            if (do_b) {
                v.x = fmaf(hdt * im, f.x, v.x);
                v.y = fmaf(hdt * im, f.y, v.y);
                v.z = fmaf(hdt * im, f.z, v.z);
            }
            if (do_a) {
                v.x = fmaf(hdt * im, f.x, v.x);
                v.y = fmaf(hdt * im, f.y, v.y);
                v.z = fmaf(hdt * im, f.z, v.z);
                x.x = fmaf(hdt, v.x, x.x);
                x.y = fmaf(hdt, v.y, x.y);
                x.z = fmaf(hdt, v.z, x.z);
                const uint4 rb = philox4x32_10(make_uint4((uint32_t)a, rep_ids[r], (uint32_t)step, 0u),
                                               P.key0, P.key1);
                const float4 xi = normals4_f32(rb);
                const float sd = tp.noise_sd[a];
                v.x = fmaf(P.c1, v.x, sd * xi.x);
                v.y = fmaf(P.c1, v.y, sd * xi.y);
                v.z = fmaf(P.c1, v.z, sd * xi.z);
                x.x = fmaf(hdt, v.x, x.x);
                x.y = fmaf(hdt, v.y, x.y);
                x.z = fmaf(hdt, v.z, x.z);
                if (!(isfinite(x.x) && isfinite(x.y) && isfinite(x.z) && isfinite(v.x) &&
                      isfinite(v.y) && isfinite(v.z)))
                    atomicOr(&st.status[r], SCPS_FLAG_NONFINITE);
                B.pos[base + s] = x;
                const float4 p0 = B.pos_ref[base + s];
                const float ddx = x.x - p0.x, ddy = x.y - p0.y, ddz = x.z - p0.z;
                d2 = fmaf(ddx, ddx, fmaf(ddy, ddy, ddz * ddz));
            }
            B.vel[base + s] = v;
        }
    }
    if (do_a) {  // non-negative floats order as unsigned
        const unsigned m = __reduce_max_sync(kFullB, __float_as_uint(d2));
        if ((threadIdx.x & 31) == 0 && m != 0u) atomicMax(&B.maxd2[r], m);
    }
}

// Frame output of the evaluated configuration (positions in atom-id order).
__global__ void k_box_frame(BoxDev B, StateDev st, RunParams P, long long frame_atoms) {
    const int r = blockIdx.y;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= B.np) return;
    const int a = B.id[(size_t)r * B.np + s];
    if (a < 0) return;
    const long long slot = st.n_saved[r] % P.max_frames;
    const float4 x = B.pos[(size_t)r * B.np + s];
    float* fr = st.frames + 3 * ((long long)r * frame_atoms + slot * B.n_atoms + a);
    fr[0] = x.x;
    fr[1] = x.y;
    fr[2] = x.z;
}

// Frame scalars; the potential energy is the fixed-point pair energy (2^-18 units, cleared
// here) plus the bonded energy.
__global__ void k_box_frame_scalars(BoxDev B, StateDev st, RunParams P, int R) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const long long slot = st.n_saved[r] % P.max_frames;
    const long long fi = (long long)r * P.max_frames + slot;
    st.fz[fi] = st.z[r];
    st.fzm[fi] = st.zm[r];
    st.fe[fi] = (double)B.epair[r] * 3.814697265625e-06 + B.eb[r];  // 2^-18
    st.fT[fi] = st.T[r];
    st.n_saved[r] += 1;
    B.epair[r] = 0;
}

__global__ void k_box_step_count(StateDev st, int R, long long k) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < R && st.status[r] == 0) st.step[r] += k;
}

// ------------------------------------------------------------------ host side
size_t box_chain_smem(int n_chain, int n_contacts) {
    return sizeof(float4) * n_chain + sizeof(long long) * 3 * n_chain + sizeof(float) * n_contacts;
}

// The rebuild kernels after the decision (each returns at once for a replica that does not
// rebuild), for replicas [r0, r0 + nr).
static void box_rebuild(const BoxDev& B, const TopoDev* topo, const StateDev& st, int r0, int nr,
                        cudaStream_t s) {
    k_box_key<<<dim3((B.np + 255) / 256, nr), 256, 0, s>>>(B, r0);
    k_box_scan<<<nr, kSortThreads, 0, s>>>(B, r0);
    k_box_scatter<<<dim3((B.n_atoms + 255) / 256, nr), 256, 0, s>>>(B, r0);
    k_box_keyorder<<<dim3((B.ncol * B.ncol * B.nz + 255) / 256, nr), 256, 0, s>>>(B, r0);
    const dim3 gt((B.nt + 3) / 4, nr);       // one warp per tile
    const dim3 gg((4 * B.nt + 3) / 4, nr);   // one warp per 8-slot i cluster
    k_box_subsort<<<gt, 128, 0, s>>>(B, topo, r0);
    k_box_tiles<<<gt, 128, 0, s>>>(B, topo, r0);
    k_box_list<<<gg, 128, 0, s>>>(B, st, r0);
}

// Pair forces of replicas [r0, r0 + nr).
static void box_pairs_launch(const BoxDev& B, const TopoDev* topo, const RunParams& P, int r0, int nr,
                             int elec, bool energy, cudaStream_t s) {
    const dim3 gg((4 * B.nt + 3) / 4, nr);
#define PAIRS(E)                                                                                \
    switch (elec) {                                                                             \
        case ELEC_DDIEL: k_box_pairs<ELEC_DDIEL, E><<<gg, 128, 0, s>>>(B, topo, P, r0); break;  \
        case ELEC_RF: k_box_pairs<ELEC_RF, E><<<gg, 128, 0, s>>>(B, topo, P, r0); break;        \
        case ELEC_PLAIN: k_box_pairs<ELEC_PLAIN, E><<<gg, 128, 0, s>>>(B, topo, P, r0); break;  \
        default: k_box_pairs<ELEC_NONE, E><<<gg, 128, 0, s>>>(B, topo, P, r0); break;           \
    }
    if (energy) {
        PAIRS(true)
    } else {
        PAIRS(false)
    }
#undef PAIRS
}

// Chain terms and the ratchet of replicas [r0, r0 + nr) (independent of the pair forces: the
// integrator adds the two).
static void box_chain_launch(const BoxDev& B, const TopoDev* topo, const StateDev& st,
                             const RunParams& P, int r0, int nr, int ncon_max, bool energy,
                             int do_ratchet, int count_step, cudaStream_t s) {
    const size_t smem = box_chain_smem(B.n_chain, ncon_max);
    if (energy)
        k_box_chain<true><<<nr, 512, smem, s>>>(B, topo, st, P, r0, do_ratchet, count_step);
    else
        k_box_chain<false><<<nr, 512, smem, s>>>(B, topo, st, P, r0, do_ratchet, count_step);
}

// Pair forces, then the chain terms and the ratchet, of replicas [r0, r0 + nr).
static void box_forces(const BoxDev& B, const TopoDev* topo, const StateDev& st, const RunParams& P,
                       int r0, int nr, int elec, int ncon_max, bool energy, int do_ratchet,
                       int count_step, cudaStream_t s) {
    box_pairs_launch(B, topo, P, r0, nr, elec, energy, s);
    box_chain_launch(B, topo, st, P, r0, nr, ncon_max, energy, do_ratchet, count_step, s);
}

// One force evaluation of replicas [r0, r0 + nr): rebuild when forced (or, when
// `auto_ok`, when due), pair forces, chain terms and the ratchet.
static cudaError_t box_eval(const BoxDev& B, const TopoDev* topo, const StateDev& st,
                            const RunParams& P, int r0, int nr, int elec, int ncon_max,
                            bool energy, int do_ratchet, int count_step, int auto_ok,
                            cudaStream_t s) {
    k_box_decide<<<1, 256, 0, s>>>(B, st, r0, nr, auto_ok);
    k_box_clear_hist<<<dim3((kNumKeys + 255) / 256, nr), 256, 0, s>>>(B, r0);
    box_rebuild(B, topo, st, r0, nr, s);
    box_forces(B, topo, st, P, r0, nr, elec, ncon_max, energy, do_ratchet, count_step, s);
    return cudaGetLastError();
}

// Dynamic shared memory k_box_chain may request on the current device: the opt-in per-block
// limit less its static shared block; 0 when the device cannot be queried.
size_t box_chain_smem_limit() {
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return 0;
    size_t stat = 0;
    for (const void* k : {(const void*)k_box_chain<true>, (const void*)k_box_chain<false>}) {
        cudaFuncAttributes a;
        if (cudaFuncGetAttributes(&a, k) != cudaSuccess) return 0;
        stat = a.sharedSizeBytes > stat ? a.sharedSizeBytes : stat;
    }
    return (size_t)optin > stat ? (size_t)optin - stat : 0;
}

cudaError_t box_prepare(const BoxDev& B, int n_contacts_max) {
    const size_t smem = box_chain_smem(B.n_chain, n_contacts_max);
    cudaError_t e = cudaFuncSetAttribute(k_box_chain<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_box_chain<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return e;
}

// One MD step of replicas [0, R) as a graph: the step counters, the rebuild decision (which
// sets the graph's conditional value), the rebuild kernels inside a conditional node (run
// only when some replica rebuilds), the forces, [the frame], the B half step and, unless
// `last`, the A half step of the next one (noise counter read from the step counters),
// [the frame scalars].
static cudaError_t box_step_graph(const BoxDev& B, const TopoDev* topo, const StateDev& st,
                                  const RunParams& P, const uint32_t* rep_ids, int R, int elec,
                                  int ncon_max, bool save, bool last, long long frame_atoms,
                                  cudaStream_t cs, cudaStream_t cs2, cudaGraph_t* def,
                                  cudaGraphExec_t* exec) {
    const dim3 ga((B.np + 255) / 256, R);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e != cudaSuccess) return e;
    cudaGraphConditionalHandle h;
    e = cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return e;
    }
    k_box_step_count<<<(R + 127) / 128, 128, 0, cs>>>(st, R, 1);
    k_box_decide_graph<<<1, 256, 0, cs>>>(B, st, R, h);
    cudaStreamCaptureStatus cst;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    cudaGraphNode_t cond = nullptr;
    cudaGraphNodeParams cp = {};
    e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, nullptr, &deps, nullptr, &nd);
    if (e == cudaSuccess) {
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeIf;
        cp.conditional.size = 1;
        e = cudaGraphAddNode(&cond, g, deps, nullptr, nd, &cp);
    }
    if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(cs, &cond, nullptr, 1, cudaStreamSetCaptureDependencies);
    if (e == cudaSuccess) {
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        e = cudaStreamBeginCaptureToGraph(cs2, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            k_box_clear_hist<<<dim3((kNumKeys + 255) / 256, R), 256, 0, cs2>>>(B, 0);
            box_rebuild(B, topo, st, 0, R, cs2);
            const cudaError_t le = cudaGetLastError();
            e = cudaStreamEndCapture(cs2, &body);
            if (e == cudaSuccess) e = le;
        }
    }
    cudaEvent_t fork = nullptr, join = nullptr;
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join, cudaEventDisableTiming);
    if (e == cudaSuccess) {  // the chain terms run beside the pair forces (second branch)
        e = cudaEventRecord(fork, cs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs2, fork, 0);
        if (e == cudaSuccess) {
            box_chain_launch(B, topo, st, P, 0, R, ncon_max, save, 1, 1, cs2);
            e = cudaEventRecord(join, cs2);
        }
        if (e == cudaSuccess) {
            box_pairs_launch(B, topo, P, 0, R, elec, save, cs);
            e = cudaStreamWaitEvent(cs, join, 0);
        }
    }
    if (e == cudaSuccess) {
        if (save) k_box_frame<<<ga, 256, 0, cs>>>(B, st, P, frame_atoms);
        k_box_integrate<<<ga, 256, 0, cs>>>(B, topo, st, P, rep_ids, 0, 1, last ? 0 : 1, 1);
        if (save) k_box_frame_scalars<<<(R + 127) / 128, 128, 0, cs>>>(B, st, P, R);
        e = cudaGetLastError();
    }
    cudaGraph_t out = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(cs, &out);
    if (e == cudaSuccess) e = ce;
    if (fork) cudaEventDestroy(fork);
    if (join) cudaEventDestroy(join);
    if (e == cudaSuccess) e = cudaGraphInstantiate(exec, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return e;
    }
    *def = g;
    return cudaSuccess;
}

void BoxGraphs::reset() {
    for (int v = 0; v < 4; ++v) {
        if (exec[v]) cudaGraphExecDestroy(exec[v]);
        if (def[v]) cudaGraphDestroy(def[v]);
        exec[v] = nullptr;
        def[v] = nullptr;
    }
}

// n_steps steps of replicas [0, R) on stream s: the current configuration is evaluated
// again (no scheduled rebuild here, so the result does not depend on how steps are split into
// calls) and its A half step taken; then every step is one launch of a step graph from G
// (regular, last, save, save and last; captured on first use), or, without G, the same
// kernels launched one by one.
cudaError_t box_run(const BoxDev& B, const TopoDev* topo, const StateDev& st, const RunParams& P,
                    const uint32_t* rep_ids, int R, int elec, int ncon_max, long long step0,
                    long long n_steps, long long frame_atoms, BoxGraphs* G, cudaStream_t s) {
    const dim3 ga((B.np + 255) / 256, R);
    cudaError_t e = box_eval(B, topo, st, P, 0, R, elec, ncon_max, false, 1, 0, 0, s);
    if (e != cudaSuccess) return e;
    k_box_integrate<<<ga, 256, 0, s>>>(B, topo, st, P, rep_ids, step0, 0, 1, 0);
    for (long long k = 1; k <= n_steps; ++k) {
        const long long step = step0 + k;
        const bool save = P.save_interval > 0 && step % P.save_interval == 0;
        const bool last = k == n_steps;
        if (G) {
            const int v = (save ? 2 : 0) + (last ? 1 : 0);
            if (!G->exec[v]) {
                e = box_step_graph(B, topo, st, P, rep_ids, R, elec, ncon_max, save, last,
                                   frame_atoms, G->cap, G->cap2, &G->def[v], &G->exec[v]);
                if (e != cudaSuccess) return e;
            }
            e = cudaGraphLaunch(G->exec[v], s);
            if (e != cudaSuccess) return e;
            continue;
        }
        k_box_step_count<<<(R + 127) / 128, 128, 0, s>>>(st, R, 1);
        e = box_eval(B, topo, st, P, 0, R, elec, ncon_max, save, 1, 1, 1, s);
        if (e != cudaSuccess) return e;
        if (save) k_box_frame<<<ga, 256, 0, s>>>(B, st, P, frame_atoms);
        k_box_integrate<<<ga, 256, 0, s>>>(B, topo, st, P, rep_ids, step, 1, last ? 0 : 1, 0);
        if (save) k_box_frame_scalars<<<(R + 127) / 128, 128, 0, s>>>(B, st, P, R);
    }
    return cudaGetLastError();
}

// Energy and forces of one configuration X (atom order) in the evaluation slot r_eval.
__global__ void k_box_load_frame(BoxDev B, const TopoDev* __restrict__ topo, StateDev st,
                                 const float* __restrict__ X, int r) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= B.np) return;
    const size_t base = (size_t)r * B.np;
    if (s < B.n_atoms) {
        B.pos[base + s] = make_float4(X[3 * s], X[3 * s + 1], X[3 * s + 2], topo->qs[s]);
        B.vel[base + s] = make_float4(0.f, 0.f, 0.f, 0.f);
        B.id[base + s] = s;
        B.slot_of[(size_t)r * B.n_atoms + s] = s;
    } else {
        B.id[base + s] = -1;
    }
    if (s == 0) {
        B.need[r] = 1;
        st.status[r] = 0;
    }
}

cudaError_t box_load(const BoxDev& B, const TopoDev* topo, const StateDev& st, const float* X,
                     int r, cudaStream_t s) {
    k_box_load_frame<<<(B.np + 255) / 256, 256, 0, s>>>(B, topo, st, X, r);
    return cudaGetLastError();
}

// Forces of the evaluation slot r in atom order (F may be NULL: the j parts are
// cleared all the same).
__global__ void k_box_store_forces(BoxDev B, int r, float* __restrict__ F) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= B.np) return;
    const size_t base = (size_t)r * B.np;
    float4 f = take_nb_force(B, r, s);
    const int a = B.id[base + s];
    if (a < 0 || !F) return;
    if (a < B.n_chain) {
        const float4 c = B.fch[(size_t)r * B.n_chain + a];
        f.x += c.x;
        f.y += c.y;
        f.z += c.z;
    }
    F[3 * a] = f.x;
    F[3 * a + 1] = f.y;
    F[3 * a + 2] = f.z;
}

__global__ void k_box_store_energy(BoxDev B, StateDev st, int r, double* U, double* Z) {
    *U = (double)B.epair[r] * 3.814697265625e-06 + B.eb[r];  // 2^-18
    B.epair[r] = 0;
    if (Z) *Z = st.z[r];
}

cudaError_t box_energy_forces(const BoxDev& B, const TopoDev* topo, const StateDev& st,
                              const RunParams& P, int r_eval, int elec, int ncon_max,
                              const float* X, double* U, float* F, double* Z, cudaStream_t s) {
    const int g = (B.np + 255) / 256;
    k_box_load_frame<<<g, 256, 0, s>>>(B, topo, st, X, r_eval);
    cudaError_t e = box_eval(B, topo, st, P, r_eval, 1, elec, ncon_max, true, 0, 0, 0, s);
    if (e != cudaSuccess) return e;
    k_box_store_forces<<<g, 256, 0, s>>>(B, r_eval, F);
    k_box_store_energy<<<1, 1, 0, s>>>(B, st, r_eval, U, Z);
    return cudaGetLastError();
}

}  // namespace scps
