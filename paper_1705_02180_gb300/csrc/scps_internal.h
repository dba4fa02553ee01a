// Internal data layout of the rMD engine (device tables and launch plans).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "scps_device.cuh"

namespace scps {

constexpr int kTile = 32;            // atoms per tile (one warp lane per atom)
constexpr int kMaxChainAtoms = 2048; // resident-form limit per replica (shared memory)
constexpr int kExclWindow = 32;      // excluded pairs must satisfy |i - j| < 32

// replica status bits (the values of SCPS_REPLICA_* in scps.h)
#define SCPS_FLAG_NONFINITE 1
#define SCPS_FLAG_FORCE_RANGE 2
#define SCPS_FLAG_LIST_OVERFLOW 4

// Per-topology tables in device memory (shared by all replicas of a topology).
struct TopoDev {
    int n_atoms, n_tiles;
    const float2* lj;          // (sigma/2, sqrt(24 eps))
    const float* qs;           // scaled charge (see pair_s)
    const float* inv_m;        // 1/m
    const float* noise_sd;     // sqrt((1 - c1^2) kT / m), c1 = exp(-gamma dt)
    const unsigned long long* excl;  // bit (j - i + 32) set when pair (i, j) is excluded
    int n_bonds;
    const int2* bond_ij;
    const float2* bond_par;    // (b0, kb)
    int n_angles;
    const int4* ang_ijk;       // (i, centre j, k, -)
    const float2* ang_par;     // (th0, kth)
    int n_contacts;
    const int2* con_ij;        // native-contact pairs of z(X)
    const float2* con_C0;      // C0 as float-float (hi, lo)
    const int* con_off;        // n_atoms + 1 offsets into con_nbr
    const int2* con_nbr;       // per atom: (contact index, partner atom)
    const float* tube_A;       // tube bias: average contact maps <C(t'_k)>, stored [item of
                               // kTubeItem contacts][K][contact of the item], zero-padded
    float tube_inv_n0;         // tube bias: 1 / sum_p C0_p^2 (the norm of Eq. sX)
};

constexpr int kMaxTubeK = 128;  // reference slices of the contact-map tube bias
constexpr int kTubeItem = 8;    // contacts per work item of the tube passes (and of the
                                // blocks in which the reference maps are stored)
constexpr int kMaxThreadsPair = 768;  // threads per CTA of a 2-CTA cluster (80 registers each)

// Per-replica addressing.
struct RepDev {
    int topo;
    int atom_off;     // offset into the packed per-atom state arrays
    long long frame_off;  // offset (in atoms) of the replica's frame ring buffer
    uint32_t rep_id;  // global replica id (noise counter word)
    int index;        // index of the replica in the per-replica state arrays
    long long list_off;   // byte offset of the replica's pair-list slab (resident chains)
};

// Pair list of a chain replica in global memory (one slab per replica, laid out for a
// launch with nta atom slots, nbs = nta / 8 blocks of 8 atoms):
//   j entries (uint16): for block I, the atoms j of later blocks within the list radius
//     of some atom of the block, ascending, padded to a multiple of 8 with the sentinel
//     slot nta; block I owns 8 (nbs - 1 - I) entries from offset list_jl_off(nbs, I);
//   item tables (uint32), one per CTA of a cluster: (I << 17 | near << 16 | chunk);
//   exclusion masks (uint64), one per item of those tables: bit 8 s + t set when chunk entry s
//     and block atom s ^ t form an excluded pair (items near their block only).
__host__ __device__ __forceinline__ long long list_jl_off(int nbs, int I) {
    return 8ll * ((long long)I * (nbs - 1) - (long long)I * (I - 1) / 2);
}
__host__ __device__ __forceinline__ long long list_jl_bytes(int nbs) {
    return ((2ll * 4ll * nbs * (nbs - 1)) + 15) & ~15ll;
}
__host__ __device__ __forceinline__ long long list_items_cap(int nbs) {
    return (long long)nbs * (nbs - 1) / 2 + 8;
}
__host__ __device__ __forceinline__ long long list_items_bytes(int nbs) {
    return (4 * list_items_cap(nbs) + 15) & ~15ll;
}
__host__ __device__ __forceinline__ long long list_slab_bytes(int nta) {
    const int nbs = nta / 8;
    return list_jl_bytes(nbs) + 2 * list_items_bytes(nbs) + 2 * 8 * list_items_cap(nbs);
}

// Replica state and outputs (device pointers).
struct StateDev {
    float4* x;        // packed positions (x, y, z, -)
    float4* v;        // packed velocities
    double* zm;       // running minimum of z
    double* z;        // z of the current configuration
    long long* step;  // global step counter
    double* T;        // bias functional accumulator
    int* status;      // SCPS_REPLICA_* bits
    // path output (ring buffers of max_frames per replica)
    float* frames;    // frame_off * 3 floats per replica start
    double* fz;
    double* fzm;
    double* fe;
    double* fT;
    long long* n_saved;
    // two-dimensional model state
    double2* xy;
    double* sm;       // running minimum of s_lambda (tube bias)
    double* wm;       // running minimum of w_lambda (tube bias)
    long long* pair_slots;  // resident chains: pairs one evaluation takes with the latest list
    int* list_builds;       // resident chains: pair-list builds in the latest launch
};

struct RunParams {
    int n_replicas;
    float dt, half_dt, c1;        // c1 = exp(-gamma dt)
    double k_R;
    int bias;                     // 0 none, 1 contacts, 2 toy
    float inv_r0sq;               // 1 / r0^2 (FP32)
    ff inv_r0sq_ff;               // 1 / r0^2 (float-float)
    uint32_t key0, key1;
    int save_interval, max_frames;
    long long n_steps;            // steps in this launch
    PairConst pc;
    // pair list of the resident chain kernels
    unsigned char* list_base;     // slabs (RepDev::list_off, or one per frame cluster)
    long long list_slab;          // bytes per frame cluster (frame evaluation)
    float rlist2;                 // (cutoff + skin)^2
    float skin_half;              // rebuild once the displacement bound reaches skin / 2
    int rebuild_every;            // and at least every this many steps (0: bound only)
    // two-dimensional models
    double toy_dt_over_gamma, toy_sd, toy_x_ref;
    double gamma;
    int toy_model;                // 0: double well, 1: asymmetric funnel (Eq. U, Table 1)
    // tube variables s_lambda, w_lambda on a reference path (two-dimensional models)
    int tube_k;                   // reference points
    const double2* tube_ref;      // [tube_k] points of the reference path
    const double* tube_time;      // [tube_k] their times t'
    double tube_lambda, tube_ks, tube_kw, tube_t;  // lambda, k_s, k_w, path duration t
};

// Periodic-box state of all replicas (slot arrays are [replica][np], in tile order).
struct BoxDev {
    int n_atoms, n_chain, np, nt, max_ent, rebuild_every;
    int ncol, nz;     // ncol x ncol columns in (x, y), nz bins in z per column
    float L, invL, rlist2, skin2_quarter;
    float4* pos;      // (x, y, z, qs)
    float4* vel;
    float2* par;      // (sigma/2, sqrt(24 eps))
    int* id;          // atom id of each slot, -1 for padding
    int* id2;         // sort buffer of id
    long long* facc;  // [replica][3][np] non-bonded force on the slot, fixed point 2^-20
                      // (order-free sums; cleared by whoever consumes it)
    long long* epair; // [replica] pair energy of energy evaluations, fixed point 2^-18
                      // (cleared by whoever consumes it)
    float4* pos2;     // sort buffers
    float4* vel2;
    int* slot_of;     // [replica][n_atoms]
    int* key;
    int* hist;        // [replica][8192] key counts, then running cursors (rebuild)
    int* colinfo;     // [replica][2][257] first compact position and first tile per column
    float4* pos_ref;  // positions at the last rebuild
    float4* clo;      // [replica][4 nt] boxes of the 8-slot clusters (clo.w: 1 = reference LJ only)
    float4* chi;
    uint32_t* ent;    // [replica][4 nt][max_ent] pair list of each 8-slot i cluster c: its own 8
                      // slots, then the slots j of clusters after c within r_list of some atom
                      // of c, ascending, padded to a multiple of 8 with kBoxNoSlot; an entry is
                      // j | (periodic shift + 1 per axis, 2 bits each) << 24 | 1 << 30 when j
                      // has the reference LJ parameters
    int* nent;        // [replica][4 nt] entries of each cluster (a multiple of 8)
    int* cflag;       // [replica][4 nt] per i cluster: 1 = it holds chain atoms, 2 = some entry
                      // needs the per-pair minimum image (the entry's shift may not hold for
                      // every pair until the next rebuild), 4 = all its atoms have the
                      // reference LJ parameters (the last atom's)
    int* need;        // [replica] rebuild flag
    int* since;       // [replica] evaluations since the last rebuild
    int* nbuild;      // [replica] list builds since the start of the latest step call
    int* nevent;      // [1] steps of the latest step call whose graph ran the rebuild kernels
    unsigned* maxd2;  // [replica] largest squared displacement since then (float bits)
    float4* fch;      // [replica][n_chain] bonded + bias force on chain atoms
    double* eb;       // [replica] bonded energy (save steps)
};

constexpr uint32_t kBoxNoSlot = 0x7fffffu;  // padding entry of a box pair list

// Step graphs of the periodic box (variants: regular, last step of a call, save step, save
// and last), captured on first use with the system's capture streams; they hold the box
// parameters by value, so any change of those drops them.
struct BoxGraphs {
    cudaGraphExec_t exec[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaGraph_t def[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaStream_t cap = nullptr, cap2 = nullptr;  // owned by the system
    void reset();
};

}  // namespace scps
