/*
 * scps.h - C ABI of the GB300 engine for ratchet-and-pawl biased Langevin
 * trajectories (rMD), the data-parallel hot path of Self-Consistent Path
 * Sampling (Orioli, a Beccara, Faccioli, arXiv:1705.02180).
 *
 * The library advances many independent replicas of one or more molecular
 * topologies (or of the two-dimensional double-well model) under
 *   - the Langevin equation, Eq. (Lang), integrated with BAOAB (underdamped)
 *     or Euler-Maruyama (overdamped);
 *   - a force field -grad U (bonds, angles, Lennard-Jones, Coulomb with a
 *     distance-dependent dielectric, reaction field or plain form; shifted
 *     force at the cutoff);
 *   - the ratchet-and-pawl bias of Eq. (FrMD) on the native-contact
 *     coordinate z(X) of Eq. (zrMD), built from the contact-map entries of
 *     Eq. (Cij), with z_m the running minimum of z and z_m(0) = z(X(0)).
 *
 * Conventions for every entry point:
 *   - return value: SCPS_OK (0) or a negative SCPS_ERR_* code; nothing throws
 *     or aborts; scps_last_error() gives a thread-local message for the last
 *     failure on the calling thread;
 *   - "host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *     global memory of the device the system was created on; buffers passed in
 *     are owned by the caller and only read or written during the call (or, for
 *     stream-ordered calls, until the work enqueued on `stream` completes);
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream); stream-ordered calls return after enqueueing;
 *   - units: nm, ps, amu, kJ/mol, elementary charge; forces in kJ mol^-1 nm^-1.
 */
#ifndef SCPS_H
#define SCPS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ----------------------------------------------------------------- status */
#define SCPS_OK 0
#define SCPS_ERR_INVALID_ARG (-1)   /* bad pointer, size, index or option */
#define SCPS_ERR_CUDA (-2)          /* a CUDA call failed (message has the CUDA error) */
#define SCPS_ERR_NONFINITE (-3)     /* a replica produced a non-finite force or position */
#define SCPS_ERR_LIST_OVERFLOW (-4) /* a capacity (tiles, lists, frames) was exceeded */
#define SCPS_ERR_TIMEOUT (-5)       /* a bounded device wait gave up */
#define SCPS_ERR_STATE (-6)         /* call not valid in the current state */
#define SCPS_ERR_UNSUPPORTED (-7)   /* combination of options not implemented */

/* per-replica status bits reported by scps_get_status */
#define SCPS_REPLICA_OK 0
#define SCPS_REPLICA_NONFINITE 1    /* non-finite position/velocity: replica frozen */
#define SCPS_REPLICA_FORCE_RANGE 2  /* a force partial exceeded the fixed-point range */
#define SCPS_REPLICA_LIST_OVERFLOW 4 /* periodic box: a tile had more j clusters than the list holds */

/* ----------------------------------------------------------------- enums */
enum { SCPS_MODEL_CHAIN = 0,
       SCPS_MODEL_TOY2D = 1,     /* U = (x^2 - 1)^2 + y^2, one particle per replica */
       SCPS_MODEL_FUNNEL2D = 2   /* the asymmetric funnel of Eq. (U) with the parameters of
                                    Table 1 (Sec. "Diffusion in a 2-dimensional asymmetric
                                    funnel"), one particle per replica */ };
enum { SCPS_ELEC_NONE = 0, SCPS_ELEC_DDIEL = 1, SCPS_ELEC_RF = 2, SCPS_ELEC_PLAIN = 3 };
enum { SCPS_INT_BAOAB = 0, SCPS_INT_EM = 1 };
/* execution form of scps_step_replicas:
 *   RESIDENT: every replica stays on chip for the whole call (one CTA or one
 *     CTA cluster per replica, all replicas in one launch, CUDA graph);
 *   PLAIN: reference form - one replica per kernel launch per step, FP32 float
 *     atomics in global memory, no graph. Same physics, same noise. */
enum { SCPS_EXEC_RESIDENT = 0, SCPS_EXEC_PLAIN = 1 };
enum { SCPS_BIAS_NONE = 0,
       SCPS_BIAS_RMD_CONTACTS = 1,  /* chains: ratchet of Eq. (FrMD) on z(X) of Eq. (zrMD) */
       SCPS_BIAS_RMD_TOY = 2,       /* two-dimensional models: ratchet on z = (x - x_ref)^2 */
       SCPS_BIAS_RMD_RADIAL = 3,    /* two-dimensional models: ratchet on z = sqrt(x^2 + y^2) */
       SCPS_BIAS_TUBE = 4           /* the self-consistent rMD forces F^s and F^w of Eq. (Fs)
                                       and Eq. (Fw) on the tube variables s_lambda and w_lambda
                                       of a reference path (Eq. sX, Eq. wX with the average path
                                       in place of the instantaneous one): configuration-space
                                       distance for the two-dimensional models, contact-map
                                       distance for chains */ };
enum { SCPS_ZM_FROM_X = 0, SCPS_ZM_VALUE = 1 };

/* ----------------------------------------------------------------- descriptors */
typedef struct {
    int32_t n_atoms;
    const double* mass;     /* host, n_atoms */
    const double* charge;   /* host, n_atoms */
    const double* sigma;    /* host, n_atoms; LJ sigma_ij = (sigma_i + sigma_j) / 2 */
    const double* eps;      /* host, n_atoms; LJ eps_ij = sqrt(eps_i eps_j) */
    int32_t n_bonds;
    const int32_t* bonds;   /* host, n_bonds x 2; U = kb/2 (r - b0)^2 */
    const double* b0;
    const double* kb;
    int32_t n_angles;
    const int32_t* angles;  /* host, n_angles x 3, centre atom in the middle; U = kth/2 (th - th0)^2 */
    const double* th0;      /* rad */
    const double* kth;
    int32_t n_excl;
    const int32_t* excl;    /* host, n_excl x 2 pairs left out of the non-bonded sum;
                               every excluded pair must satisfy |i - j| < 32 */
} scps_topology_desc;

typedef struct {
    int32_t model;                          /* SCPS_MODEL_* */
    int32_t n_topologies;                   /* chain model: >= 1; toy: 0 */
    const scps_topology_desc* topologies;   /* host, n_topologies */
    int32_t n_replicas;
    const int32_t* replica_topology;        /* host, n_replicas (chain model) */
    const int32_t* replica_id;              /* host, n_replicas global ids for the noise counter;
                                               NULL = 0 .. n_replicas-1 */
    const double* x0;   /* host, packed: replicas in order, n_atoms(topology) x 3 each (toy: x 2) */
    const double* v0;   /* host, same layout as x0; NULL = zero (ignored by SCPS_INT_EM) */
    /* non-bonded */
    double cutoff;      /* nm */
    int32_t elec;       /* SCPS_ELEC_* */
    double k_dd;        /* distance-dependent dielectric eps_r = k_dd r (nm^-1), e.g. 40 */
    double eps_rf;      /* reaction-field dielectric, e.g. 78.5 */
    double box;         /* 0: open boundaries; > 0: cubic periodic box of this edge (nm), with
                           minimum-image bonded terms and contacts, column-sorted tiles and
                           cluster pair lists (one topology; its bonded atoms, the "chain", come
                           first; the remaining atoms are solvent sites). Reaction field is the
                           intended electrostatics. Needs box > 2 (cutoff + skin). */
    /* integrator */
    int32_t integrator; /* SCPS_INT_* */
    double dt, gamma, kT;
    uint64_t seed;      /* Philox4x32-10 key */
    /* path output */
    int32_t save_interval;  /* global steps between saved frames; 0 = no frames */
    int32_t max_frames;     /* frames kept per replica (the oldest are overwritten) */
    /* execution */
    int32_t exec;           /* SCPS_EXEC_* */
    int32_t cluster_size;   /* CTAs per replica in RESIDENT form: 0 = auto, 1 or 2 */
    int32_t threads;        /* threads per CTA in RESIDENT form: 0 = auto, else 128..1024
                               (at most 768 with cluster_size 2) */
    int32_t steps_per_graph;/* device-loop steps per CUDA-graph node: 0 = auto */
    /* pair lists */
    double skin;            /* list buffer r_list - r_c (nm); 0 = default (0.15 for the periodic
                               box, 0.12 for chains). A list is rebuilt before any pair inside
                               r_c can be missing: periodic box, once an atom has moved skin/2
                               since the last build (the lists of all live replicas are then
                               rebuilt together); chains, once a bound on every atom's
                               displacement since then (dt/2 times the largest |v| + |v'| of
                               each step, summed) reaches skin/2. Forces do not depend on the
                               skin or the rebuild cadence (chains: bit for bit). */
    int32_t rebuild_every;  /* periodic box: scheduled rebuild interval (steps), 0 = 20, all
                               live replicas together as soon as one is due; chains:
                               also rebuild at least every this many steps, 0 = only by the
                               displacement bound */
} scps_system_desc;

typedef struct {
    int32_t kind;                       /* SCPS_BIAS_* */
    double k_R;                         /* ratchet constant of Eq. (FrMD) */
    double r0;                          /* reference distance of Eq. (Cij), nm */
    const int32_t* n_pairs;             /* host, per topology: native-contact pair count */
    const int32_t* const* pairs;        /* host, per topology: n_pairs x 2 (i, j) pairs of z(X) */
    const double* const* x_native;      /* host, per topology: native coordinates n_atoms x 3;
                                           C0_ij = C_ij(X_N) is computed by the library */
    int32_t zm_init;                    /* SCPS_ZM_FROM_X: z_m = z(X) of the current state
                                           (the paper's z_m(0) = z(X(0))); SCPS_ZM_VALUE */
    double zm_value;
    double toy_x_ref;                   /* toy model: z = (x - toy_x_ref)^2 */
    /* SCPS_BIAS_TUBE: reference path <X(t'_k)>, k = 0 .. n_ref-1 (host, n_ref x 2), its
       times t'_k (host, n_ref), lambda, k_s, k_w of Eq. (Fs) and Eq. (Fw), and the path
       duration t. With D_k = |X - <X(t'_k)>|^2 and pi_k = exp(-lambda D_k) / sum:
       w = -(1/lambda) log sum_k exp(-lambda D_k), s = 1 - (1/t) sum_k t'_k pi_k. s_m and
       w_m are their running minima (zm_init as for z_m). */
    int32_t n_ref;
    const double* ref;
    const double* ref_time;
    double lambda, k_s, k_w, t_path;
    /* SCPS_BIAS_TUBE on chains (resident form): per topology (host) the average contact maps
       <C_p(t'_k)> over the topology's native-contact list (the pairs and x_native above),
       n_ref x n_pairs[t], slice-major. D_k = sum_p (C_p(X) - <C_p(t'_k)>)^2 / sum_p C0_p^2
       replaces |X - <X(t'_k)>|^2; n_ref <= 128. */
    const double* const* ref_maps;
} scps_bias_desc;

typedef struct {
    int32_t n_replicas;
    int64_t n_atoms_total;              /* sum over replicas */
    int32_t max_atoms;
    int32_t cluster_size, threads, steps_per_graph;
    int32_t kernels_per_step_call;      /* kernel launches one scps_step_replicas call enqueues
                                           per graph node (resident form) */
    int64_t graph_nodes_last_call;      /* kernel launches enqueued by the last step call
                                           (periodic box: including the 8 rebuild kernels of
                                           each step that rebuilt; synchronises) */
    int64_t pair_checks_per_step;       /* resident chains: non-bonded pair slots one step
                                           evaluates, summed over replicas, with the pair list
                                           each replica built last (64 per list item of 8 x 8
                                           atoms, 28 per block of 8 with itself); periodic
                                           box: 64 per chunk of 8 list entries of an 8-slot
                                           cluster (synchronises) */
    size_t device_bytes;                /* device memory held by the system */
    int32_t launch_groups;              /* resident form: launches per step call chunk */
    int32_t plan;                       /* resident form: SCPS_PLAN_* */
    double list_skin;                   /* pair-list skin r_list - r_c (nm) */
    double steps_per_list_build;        /* resident chains: mean steps per pair-list build in
                                           the latest launch (the build that opens a launch
                                           counts); periodic box: mean steps per list build
                                           of a replica in the latest step call */
} scps_info;

/* launch plans of the resident form */
enum { SCPS_PLAN_ONE_LAUNCH = 0,        /* one launch, replicas by decreasing size */
       SCPS_PLAN_PER_SIZE_CLASS = 1 };  /* one launch per size class (tile-rounded atom
                                           count), shared memory sized per class, the
                                           launches running side by side */

typedef struct {
    int32_t plan;                       /* chosen SCPS_PLAN_* */
    int32_t cluster_size, threads;      /* chosen CTAs per replica and threads per CTA */
    int32_t candidates;                 /* configurations timed (0 when taken from the cache) */
    int32_t from_cache;                 /* 1: the choice came from the process-wide cache */
    double us_per_step;                 /* probe time per step of the choice */
    double us_per_step_initial;         /* probe time per step of the configuration before */
    double skin;                        /* chosen pair-list skin (nm) */
    int32_t rebuild_every;              /* periodic box: chosen rebuild cadence (steps);
                                           chains: the descriptor's value (0: displacement only) */
} scps_tune_result;

typedef struct scps_system scps_system;

/* ----------------------------------------------------------------- entry points */
/* Creates a system on the current CUDA device: copies every descriptor array
 * (the caller keeps ownership), allocates state, frames and topology tables in
 * device memory. Velocities default to zero. No bias until scps_set_bias. */
int scps_create_system(const scps_system_desc* d, scps_system** out);

/* Frees all device and host memory of the system (NULL is ignored). */
int scps_destroy_system(scps_system* s);

/* Sets the ratchet bias of Eq. (FrMD) on z(X) of Eq. (zrMD) (contact-map form)
 * or on z = (x - x_ref)^2 (toy). Computes C0_ij = C_ij(X_N) per topology and
 * resets z_m per replica (SCPS_ZM_FROM_X uses the current positions). Clears
 * the bias-functional accumulators. Synchronous. */
int scps_set_bias(scps_system* s, const scps_bias_desc* b);

/* Advances every replica by n_steps steps (rMD: forces, z, ratchet, update,
 * frame output). Stream-ordered on `stream`; returns after enqueueing. Device
 * errors of the enqueued work are reported by scps_get_status.
 * Chains (RESIDENT form): one launch per group and chunk of steps_per_graph steps, each a
 * CUDA graph captured on first use; the pair lists are built inside the kernel.
 * Periodic box: the call first evaluates the current configuration again (no scheduled
 * rebuild, so the split of steps into calls does not change results), then runs every step
 * as one CUDA graph whose pair-list rebuild sits in a conditional node that runs only when
 * some replica's rebuild is due (it then rebuilds the lists of all live replicas); the step
 * counters advance one step at a time (a replica
 * frozen by an error keeps the count it had). */
int scps_step_replicas(scps_system* s, int64_t n_steps, void* stream);

/* Potential energy, forces and z for n_frames configurations of topology
 * `topo` (no bias force, no state change). X: device float, n_frames x
 * n_atoms x 3. U: device double, n_frames (total physical energy). F: device
 * float, n_frames x n_atoms x 3, may be NULL. z: device double, n_frames, may
 * be NULL (needs the contact list of a contact or tube bias). Stream-ordered. Each frame's
 * pair list is built in a scratch owned by the system (grown, with a device synchronisation,
 * when a call needs more frames per launch than any before): calls of one system on
 * different streams must not overlap in time (order them with events, or use one stream);
 * scps_hvp uses no such scratch. */
int scps_energy_forces(scps_system* s, int32_t topo, int64_t n_frames, const float* X,
                       double* U, float* F, double* z, void* stream);

/* Hessian-vector products H(X_t) V_t of the physical potential for n_frames
 * frames (device float arrays n_frames x n_atoms x 3). Stream-ordered. The gradient
 * of sum_t |grad U(X_t)|^2, a term of the Onsager-Machlup action of Eq. (SOM), is
 * sum_t 2 H(X_t) grad U(X_t). Open-boundary chains only: a periodic-box system gets
 * SCPS_ERR_UNSUPPORTED. Pair terms are summed per item in FP32, then in fixed point. */
int scps_hvp(scps_system* s, int32_t topo, int64_t n_frames, const float* X, const float* V,
             float* HV, void* stream);

/* Copies saved path frames of replicas [rep0, rep0 + nrep) to host buffers,
 * oldest first (synchronous). frames: float, per replica max_frames x
 * n_atoms x 3 packed in replica order (toy: x 2); z, zmin, epot, bias_T:
 * double, per replica max_frames; n_frames_out: per replica count (<=
 * max_frames). Any output pointer may be NULL. */
int scps_collect_paths(scps_system* s, int32_t rep0, int32_t nrep, float* frames, double* z,
                       double* zmin, double* epot, double* bias_T, int64_t* n_frames_out);

/* Checkpoint: copies (to host) or replaces (from host) the full dynamical
 * state - positions, velocities, z_m, step counters, bias functional T - in the
 * packed x0 layout (synchronous). Resuming from a saved state reproduces the
 * uninterrupted run bit for bit. Any pointer may be NULL (left unchanged). */
int scps_get_state(scps_system* s, double* x, double* v, double* zm, int64_t* step,
                   double* bias_T);
int scps_set_state(scps_system* s, const double* x, const double* v, const double* zm,
                   const int64_t* step, const double* bias_T);

/* Synchronises and returns SCPS_OK or the first error of the enqueued work:
 * SCPS_ERR_NONFINITE when a replica has the NONFINITE or FORCE_RANGE bit,
 * else SCPS_ERR_LIST_OVERFLOW when one has the LIST_OVERFLOW bit. A flagged
 * replica is frozen. per_replica (host, n_replicas, may be NULL) receives
 * the SCPS_REPLICA_* bits. */
int scps_get_status(scps_system* s, int32_t* per_replica);

/* Sizes and launch shape of the system (host `info`). Synchronises the device (it reads the
 * per-replica pair-slot counts of the last step call). */
int scps_get_info(const scps_system* s, scps_info* info);

/* Average path of selected replicas (step 3 of the SCPS iteration; Eq. avCij):
 * for the two-dimensional models, out[k] = mean over the replicas in `replicas`
 * (host, n_sel indices) of their saved frame k, k = 0 .. n_frames-1, oldest first
 * (host, n_frames x 2); for chains (one topology among the selected replicas, whose
 * contact list a contact or tube bias has set), out[k * n_pairs + p] = mean of
 * C_p of Eq. (Cij) over the selected frames k (host, n_frames x n_pairs, FP64).
 * Every selected replica must still hold all its frames (n_saved <= max_frames)
 * and have at least n_frames of them. Synchronous. */
int scps_path_average(scps_system* s, int32_t n_sel, const int32_t* replicas, int32_t n_frames,
                      double* out);

/* Autotuner of the resident form (chain replicas): times the launch plans
 * (SCPS_PLAN_*), cluster sizes {1, 2} and threads per CTA {256, 512, 1024} (768 in
 * place of 1024 for 2-CTA clusters) on the system itself, then, at the chosen shape, the
 * pair-list skin {0.06, 0.09, 0.12, 0.16, 0.2} nm (a larger skin adds pairs to every
 * step and makes list builds rarer: the rebuild cadence follows from the displacement
 * bound), probe_steps steps each from the current state (restored after every probe; no
 * frames are saved while probing), and keeps the fastest; a candidate replaces the
 * current configuration (or an earlier candidate) only when it is more than 2 % faster,
 * so timing noise does not switch shapes. The choice is cached per process under (SM
 * count, electrostatics, bias kind, multiset of replica sizes); use_cache != 0 takes a
 * cached choice without probing. The plan changes only which CTA runs which replica and
 * forces do not depend on the skin, so trajectories are bit-identical under every
 * choice.
 * Periodic box: the pair-list skin {0.1, 0.15, 0.2} nm x the rebuild cadence {10, 20,
 * 40} steps (a rebuild also comes earlier once an atom has moved skin/2), probed the
 * same way from a device snapshot of the box state; the probes and the final choice
 * force a list rebuild at the next step, so the trajectory equals that of a run with one
 * more rebuild there (positions are wrapped into the box at each rebuild: equal to
 * rounding, not bit for bit). Cached under (SM count, electrostatics, atoms, replicas).
 * Synchronous; out may be NULL. */
int scps_autotune(scps_system* s, int32_t probe_steps, int32_t use_cache, scps_tune_result* out);

/* Philox4x32-10 blocks on the device, for checking the noise stream:
 * ctr: device uint32 n x 4, key: two uint32 words, out: device uint32 n x 4. */
int scps_philox4x32_10(int64_t n, const uint32_t* ctr, uint32_t key0, uint32_t key1,
                       uint32_t* out, void* stream);

/* Allocation-free variant of scps_energy_forces for one configuration (the
 * paper has no counterpart; it serves callers that cannot allocate device
 * memory when they need forces: code running inside a CUDA stream capture,
 * where cudaMalloc is not allowed; frameworks that have reserved the device
 * memory for their own pool; latency-critical loops that must not allocate).
 * Open-boundary chain systems only: a periodic-box system returns
 * SCPS_ERR_UNSUPPORTED (these kernels take no periodic images).
 * X: device float n_atoms x 3 of topology `topo`; U: device double (1 value);
 * F: device float n_atoms x 3, may be NULL. Physical energy and forces only.
 * Forces and energy are summed in 64-bit fixed point (2^-20 units) with integer
 * atomics, so the result does not depend on thread order and repeated calls on
 * the same X return the same bits (they may differ from scps_energy_forces in
 * the last bits: the two sum their FP32 pair terms in different groups).
 * It calls no cudaMalloc/cudaFree: the kernels accumulate into a static device
 * array of this library (sized for at most 8192 atoms, held by every GPU that
 * loads the library until the process exits); larger topologies return
 * SCPS_ERR_UNSUPPORTED (chain systems are limited to 2048 atoms at creation,
 * so the check is a safeguard). Each call clears the part it uses first. All
 * calls share that array, so calls that overlap on the GPU (on different
 * streams, or from several threads) race and corrupt each other's results;
 * serialise them. The first call on a device looks up the array's device
 * address (once per device, with that device current); make that first call
 * before any stream capture. Stream-ordered on `stream`. */
int scps_energy_forces_noalloc(scps_system* s, int32_t topo, const float* X, double* U, float* F,
                               void* stream);

/* Thread-local message of the last failure on this thread ("" if none). */
const char* scps_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SCPS_H */
