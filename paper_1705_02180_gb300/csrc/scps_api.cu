// C ABI of the rMD engine (include/scps.h): validation, device tables, state,
// launch plans and CUDA graphs. All compute runs in the kernels of
// kern_chain.cu and kern_aux.cu.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <limits>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/scps.h"
#include "scps_internal.h"

namespace scps {
size_t resident_smem_bytes(int nta);
size_t resident_smem_limit();
size_t box_chain_smem_limit();
size_t box_chain_smem(int n_chain, int n_contacts);
cudaError_t launch_resident(int elec, int cluster, const TopoDev* topos, const RepDev* reps,
                            const StateDev& st, const RunParams& P, int nta, int threads,
                            cudaStream_t stream);
cudaError_t launch_eval(int elec, const TopoDev* topo, const RunParams& P, const float* X,
                        double* U, float* F, double* Z, long long n_frames, int nta, int threads,
                        int cl, cudaStream_t stream);
cudaError_t launch_path_average_2d(const StateDev& st, int max_frames, int K, const int* sel,
                                   int n_sel, double2* out, cudaStream_t stream);
cudaError_t launch_path_average_contacts(const StateDev& st, const int2* con_ij, int nc, int n,
                                         const long long* frame_off, int n_sel, int K,
                                         double inv_r0sq, double* out, cudaStream_t stream);
cudaError_t launch_toy(const StateDev& st, const RunParams& P, const uint32_t* rep_ids,
                       cudaStream_t stream);
cudaError_t launch_philox(long long n, const uint32_t* ctr, uint32_t k0, uint32_t k1,
                          uint32_t* out, cudaStream_t stream);
cudaError_t plain_run_replica(int elec, const TopoDev& tp, const StateDev& st, int r,
                              const RepDev& rep, const RunParams& P, float* scratch,
                              double* dscratch, long long step0, cudaStream_t s);
cudaError_t launch_native_map(int nc, const int2* pairs, const double* xN, double inv_r0sq,
                              float2* C0, cudaStream_t s);
cudaError_t launch_add_steps(long long* step, int n, long long k, cudaStream_t s);
cudaError_t launch_hvp(int elec, const TopoDev* topo, const RunParams& P, const float* X,
                       const float* V, float* HV, long long n_frames, int nta, cudaStream_t s);
cudaError_t box_prepare(const BoxDev& B, int n_contacts_max);
cudaError_t box_load(const BoxDev& B, const TopoDev* topo, const StateDev& st, const float* X,
                     int r, cudaStream_t s);
cudaError_t box_run(const BoxDev& B, const TopoDev* topo, const StateDev& st, const RunParams& P,
                    const uint32_t* rep_ids, int R, int elec, int ncon_max, long long step0,
                    long long n_steps, long long frame_atoms, BoxGraphs* G, cudaStream_t s);
cudaError_t box_energy_forces(const BoxDev& B, const TopoDev* topo, const StateDev& st,
                              const RunParams& P, int r_eval, int elec, int ncon_max,
                              const float* X, double* U, float* F, double* Z, cudaStream_t s);
constexpr int kMaxBoxAtoms = 1 << 20;
}  // namespace scps

using namespace scps;

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define SCPS_CU(call)                                                                     \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(SCPS_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));   \
    } while (0)

constexpr double kCoulombF = 138.935458;  // kJ mol^-1 nm e^-2
constexpr double kDefaultChainSkin = 0.12;  // nm: pair-list buffer of the chain kernels
constexpr long long kEvalFramesPerLaunch = 1024;  // frame clusters per evaluation launch

struct TopoHost {
    int n = 0, ncon = 0;
    std::vector<float> inv_m;
    TopoDev dev{};
};

}  // namespace

struct scps_system {
    int device = 0;
    int model = SCPS_MODEL_CHAIN;
    scps_system_desc d{};
    std::vector<TopoHost> topos;
    std::vector<int> rep_topo, atom_off;
    std::vector<long long> frame_off;
    std::vector<uint32_t> rep_id;
    std::vector<long long> host_step;
    long long n_atoms_total = 0, n_frame_atoms = 0;
    int max_atoms = 0, nta = 0, ncon_max = 0;
    // pair lists of the resident chain kernels: one slab per replica, and one per frame
    // cluster of the frame evaluation (grown on demand, at most kEvalFramesPerLaunch)
    unsigned char* d_lists = nullptr;
    long long list_slab = 0;
    unsigned char* d_eval_lists = nullptr;
    long long eval_frames_cap = 0, eval_slab = 0;
    double list_skin = 0.0;          // r_list - r_c of the chain pair lists
    long long last_launch_steps = 0; // steps of the latest resident launch
    TopoDev* d_topos = nullptr;
    RepDev* d_reps = nullptr;
    uint32_t* d_rep_ids = nullptr;
    StateDev st{};
    RunParams base{};
    std::vector<void*> allocs;
    cudaStream_t cap_stream = nullptr;
    BoxGraphs box_graphs;  // periodic box: step graphs and their capture streams
    std::map<long long, cudaGraphExec_t> graphs;
    std::vector<cudaGraph_t> graph_defs;
    float* plain_f = nullptr;
    double* plain_d = nullptr;
    int threads = 0, cluster = 1, steps_per_graph = 0;
    // resident form: one launch per group (groups after the first run on forked streams)
    struct Group {
        RepDev* d_reps = nullptr;  // this group's replicas (owned by `allocs`)
        int count = 0, nta = 0, cluster = 1, threads = 1024;
    };
    std::vector<Group> groups;
    int plan = 0;  // 0: one launch, replicas by decreasing size; 1: one launch per size class
    std::vector<cudaStream_t> fork_streams;
    std::vector<cudaEvent_t> fork_events;
    int bias_kind = SCPS_BIAS_NONE;
    double inv_r0sq = 0.0;  // 1 / r0^2 of the contact bias (FP64)
    scps_info info{};
    size_t bytes = 0;
    bool is_box = false;
    BoxDev box{};

    template <class T>
    cudaError_t alloc(T** p, size_t n) {
        if (n == 0) n = 1;
        cudaError_t e = cudaMalloc((void**)p, sizeof(T) * n);
        if (e == cudaSuccess) {
            allocs.push_back(*p);
            bytes += sizeof(T) * n;
            e = cudaMemset(*p, 0, sizeof(T) * n);
        }
        return e;
    }
    template <class T>
    cudaError_t upload(T** p, const std::vector<T>& h) {
        cudaError_t e = alloc(p, h.size());
        if (e == cudaSuccess && !h.empty())
            e = cudaMemcpy(*p, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice);
        return e;
    }
    // tables of the current bias: replaced (and freed) by the next scps_set_bias
    std::vector<void*> bias_allocs;
    template <class T>
    cudaError_t bias_upload(T** p, const std::vector<T>& h) {
        const size_t n = h.empty() ? 1 : h.size();
        cudaError_t e = cudaMalloc((void**)p, sizeof(T) * n);
        if (e != cudaSuccess) return e;
        bias_allocs.push_back(*p);
        if (!h.empty()) e = cudaMemcpy(*p, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice);
        return e;
    }
    void drop_bias_tables() {
        for (void* q : bias_allocs) cudaFree(q);
        bias_allocs.clear();
    }
};

namespace {

bool is_2d(int model) { return model == SCPS_MODEL_TOY2D || model == SCPS_MODEL_FUNNEL2D; }

// NVTX range around every entry point (a no-op unless a profiler is attached).
struct TraceRange {
    explicit TraceRange(const char* name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
};

int validate_topology(const scps_topology_desc& t, int idx, int max_atoms) {
    if (t.n_atoms <= 0 || t.n_atoms > max_atoms)
        return fail(SCPS_ERR_INVALID_ARG, "topology %d: n_atoms %d outside [1, %d]", idx, t.n_atoms,
                    max_atoms);
    if (!t.mass || !t.charge || !t.sigma || !t.eps)
        return fail(SCPS_ERR_INVALID_ARG, "topology %d: per-atom array is NULL", idx);
    if (t.n_bonds < 0 || t.n_angles < 0 || t.n_excl < 0)
        return fail(SCPS_ERR_INVALID_ARG, "topology %d: negative list size", idx);
    if ((t.n_bonds && (!t.bonds || !t.b0 || !t.kb)) || (t.n_angles && (!t.angles || !t.th0 || !t.kth)) ||
        (t.n_excl && !t.excl))
        return fail(SCPS_ERR_INVALID_ARG, "topology %d: list array is NULL", idx);
    const int n = t.n_atoms;
    for (int i = 0; i < n; ++i) {
        if (!(t.mass[i] > 0.0) || !std::isfinite(t.mass[i]))
            return fail(SCPS_ERR_INVALID_ARG, "topology %d: mass[%d] must be > 0", idx, i);
        if (!(t.eps[i] >= 0.0) || !(t.sigma[i] >= 0.0) || !std::isfinite(t.charge[i]))
            return fail(SCPS_ERR_INVALID_ARG, "topology %d: bad LJ/charge parameter at atom %d", idx, i);
    }
    for (int b = 0; b < t.n_bonds; ++b) {
        const int i = t.bonds[2 * b], j = t.bonds[2 * b + 1];
        if (i < 0 || j < 0 || i >= n || j >= n || i == j)
            return fail(SCPS_ERR_INVALID_ARG, "topology %d: bond %d has bad atoms (%d, %d)", idx, b, i, j);
    }
    for (int a = 0; a < t.n_angles; ++a) {
        const int i = t.angles[3 * a], j = t.angles[3 * a + 1], k = t.angles[3 * a + 2];
        if (i < 0 || j < 0 || k < 0 || i >= n || j >= n || k >= n || i == j || j == k || i == k)
            return fail(SCPS_ERR_INVALID_ARG, "topology %d: angle %d has bad atoms", idx, a);
    }
    for (int e = 0; e < t.n_excl; ++e) {
        const int i = t.excl[2 * e], j = t.excl[2 * e + 1];
        if (i < 0 || j < 0 || i >= n || j >= n || i == j)
            return fail(SCPS_ERR_INVALID_ARG, "topology %d: exclusion %d has bad atoms", idx, e);
        if (std::abs(i - j) >= kExclWindow)
            return fail(SCPS_ERR_UNSUPPORTED,
                        "topology %d: excluded pair (%d, %d) is %d apart; the limit is %d", idx, i,
                        j, std::abs(i - j), kExclWindow - 1);
    }
    return SCPS_OK;
}

int build_topology(scps_system* s, const scps_topology_desc& t, TopoHost& h) {
    const scps_system_desc& d = s->d;
    const int n = t.n_atoms;
    h.n = n;
    double qscale = 0.0;
    if (d.elec == SCPS_ELEC_DDIEL) qscale = std::sqrt(2.0 * kCoulombF / d.k_dd);
    if (d.elec == SCPS_ELEC_RF || d.elec == SCPS_ELEC_PLAIN) qscale = std::sqrt(kCoulombF);
    const double c1 = std::exp(-d.gamma * d.dt);
    std::vector<float2> lj(n);
    std::vector<float> qs(n), inv_m(n), sd(n);
    std::vector<unsigned long long> excl(n, 0ull);
    for (int i = 0; i < n; ++i) {
        lj[i] = make_float2((float)(0.5 * t.sigma[i]), (float)std::sqrt(24.0 * t.eps[i]));
        qs[i] = (float)(qscale * t.charge[i]);
        inv_m[i] = (float)(1.0 / t.mass[i]);
        sd[i] = (float)std::sqrt((1.0 - c1 * c1) * d.kT / t.mass[i]);
    }
    for (int e = 0; e < t.n_excl; ++e) {
        const int i = t.excl[2 * e], j = t.excl[2 * e + 1];
        excl[i] |= 1ull << (j - i + kExclWindow);
        excl[j] |= 1ull << (i - j + kExclWindow);
    }
    std::vector<int2> bij(t.n_bonds);
    std::vector<float2> bpar(t.n_bonds);
    for (int b = 0; b < t.n_bonds; ++b) {
        bij[b] = make_int2(t.bonds[2 * b], t.bonds[2 * b + 1]);
        bpar[b] = make_float2((float)t.b0[b], (float)t.kb[b]);
    }
    std::vector<int4> aijk(t.n_angles);
    std::vector<float2> apar(t.n_angles);
    for (int a = 0; a < t.n_angles; ++a) {
        aijk[a] = make_int4(t.angles[3 * a], t.angles[3 * a + 1], t.angles[3 * a + 2], 0);
        apar[a] = make_float2((float)t.th0[a], (float)t.kth[a]);
    }
    float2* d_lj;
    float *d_qs, *d_im, *d_sd;
    unsigned long long* d_ex;
    int2* d_bij;
    float2* d_bpar;
    int4* d_aijk;
    float2* d_apar;
    SCPS_CU(s->upload(&d_lj, lj));
    SCPS_CU(s->upload(&d_qs, qs));
    SCPS_CU(s->upload(&d_im, inv_m));
    SCPS_CU(s->upload(&d_sd, sd));
    SCPS_CU(s->upload(&d_ex, excl));
    SCPS_CU(s->upload(&d_bij, bij));
    SCPS_CU(s->upload(&d_bpar, bpar));
    SCPS_CU(s->upload(&d_aijk, aijk));
    SCPS_CU(s->upload(&d_apar, apar));
    h.inv_m = inv_m;
    TopoDev& td = h.dev;
    td.n_atoms = n;
    td.n_tiles = (n + kTile - 1) / kTile;
    td.lj = d_lj;
    td.qs = d_qs;
    td.inv_m = d_im;
    td.noise_sd = d_sd;
    td.excl = d_ex;
    td.n_bonds = t.n_bonds;
    td.bond_ij = d_bij;
    td.bond_par = d_bpar;
    td.n_angles = t.n_angles;
    td.ang_ijk = d_aijk;
    td.ang_par = d_apar;
    td.n_contacts = 0;
    td.con_ij = nullptr;
    td.con_C0 = nullptr;
    return SCPS_OK;
}

int atoms_per_replica(const scps_system* s, int r) {
    return is_2d(s->model) ? 1 : s->topos[s->rep_topo[r]].n;
}

int auto_threads(int nta) {
    if (nta <= 256) return 256;
    if (nta <= 640) return 512;
    return 1024;
}

int sync_topos(scps_system* s) {
    std::vector<TopoDev> h(s->topos.size());
    for (size_t t = 0; t < h.size(); ++t) h[t] = s->topos[t].dev;
    SCPS_CU(cudaMemcpy(s->d_topos, h.data(), sizeof(TopoDev) * h.size(), cudaMemcpyHostToDevice));
    return SCPS_OK;
}

void drop_graphs(scps_system* s) {
    s->box_graphs.reset();
    for (auto& kv : s->graphs) cudaGraphExecDestroy(kv.second);
    s->graphs.clear();
    for (auto g : s->graph_defs) cudaGraphDestroy(g);
    s->graph_defs.clear();
}

int tile_atoms(int n) { return ((n + kTile - 1) / kTile) * kTile; }

// Launch groups of the resident form. plan 0: one group, replicas by decreasing
// size (large replicas start first, small ones fill the last wave); plan 1: one
// group per size class (tile-rounded atom count), each with shared memory for its
// own size. Every group gets the given cluster size and threads per CTA.
int set_groups(scps_system* s, int plan, int cluster, int threads) {
    if (cluster == 2 && threads > kMaxThreadsPair)
        return fail(SCPS_ERR_INVALID_ARG, "a 2-CTA cluster takes at most %d threads per CTA",
                    kMaxThreadsPair);
    const int R = s->d.n_replicas;
    std::vector<int> order(R);
    for (int r = 0; r < R; ++r) order[r] = r;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return s->topos[s->rep_topo[a]].n > s->topos[s->rep_topo[b]].n;
    });
    std::vector<std::vector<int>> members;
    if (plan == 0) {
        members.push_back(order);
    } else {
        int last = -1;
        for (int r : order) {
            const int c = tile_atoms(s->topos[s->rep_topo[r]].n);
            if (c != last) members.emplace_back();
            members.back().push_back(r);
            last = c;
        }
    }
    std::vector<scps_system::Group> groups;
    for (auto& m : members) {
        scps_system::Group g;
        g.count = (int)m.size();
        int na = 0;
        for (int r : m) na = std::max(na, s->topos[s->rep_topo[r]].n);
        g.nta = plan == 0 ? s->nta : tile_atoms(na);
        g.cluster = cluster;
        g.threads = threads;
        std::vector<RepDev> reps(m.size());
        for (size_t k = 0; k < m.size(); ++k) {
            const int r = m[k];
            reps[k] = RepDev{s->rep_topo[r], s->atom_off[r], s->frame_off[r], s->rep_id[r], r,
                             (long long)r * s->list_slab};
        }
        SCPS_CU(s->upload(&g.d_reps, reps));
        groups.push_back(g);
    }
    while (s->fork_streams.size() + 1 < groups.size()) {
        cudaStream_t st;
        cudaEvent_t ev;
        SCPS_CU(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        SCPS_CU(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        s->fork_streams.push_back(st);
        s->fork_events.push_back(ev);
    }
    if (s->fork_events.size() < groups.size()) {  // one more for the fork itself
        cudaEvent_t ev;
        SCPS_CU(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        s->fork_events.push_back(ev);
    }
    s->groups = groups;
    s->plan = plan;
    s->cluster = cluster;
    s->threads = threads;
    drop_graphs(s);
    return SCPS_OK;
}

// One launch per group for n_steps steps; groups after the first run on forked
// streams that join `cs` again (also under stream capture).
cudaError_t launch_groups(scps_system* s, const RunParams& P0, long long n_steps, cudaStream_t cs) {
    const size_t G = s->groups.size();
    if (G > 1) {
        cudaError_t e = cudaEventRecord(s->fork_events[G - 1], cs);
        for (size_t k = 1; k < G && e == cudaSuccess; ++k)
            e = cudaStreamWaitEvent(s->fork_streams[k - 1], s->fork_events[G - 1], 0);
        if (e != cudaSuccess) return e;
    }
    for (size_t k = 0; k < G; ++k) {
        const scps_system::Group& g = s->groups[k];
        RunParams P = P0;
        P.n_steps = n_steps;
        P.n_replicas = g.count;
        cudaStream_t st = k == 0 ? cs : s->fork_streams[k - 1];
        cudaError_t e = launch_resident(s->d.elec, g.cluster, s->d_topos, g.d_reps, s->st, P, g.nta,
                                        g.threads, st);
        if (e != cudaSuccess) return e;
    }
    for (size_t k = 1; k < G; ++k) {
        cudaError_t e = cudaEventRecord(s->fork_events[k - 1], s->fork_streams[k - 1]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, s->fork_events[k - 1], 0);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// List radius of the resident chain kernels (forces do not depend on it: the skin only
// trades pairs per step against list rebuilds).
void set_skin(scps_system* s, double skin) {
    const double rc = s->base.pc.rc > 0.f ? (double)s->base.pc.rc : 1.0;
    s->list_skin = skin;
    s->base.rlist2 = (float)((rc + skin) * (rc + skin));
    s->base.skin_half = (float)(0.5 * skin);
}

}  // namespace

extern "C" {

const char* scps_last_error(void) { return g_err.c_str(); }

int scps_create_system(const scps_system_desc* d, scps_system** out) {
    TraceRange trace_("scps_create_system");
    if (!d || !out) return fail(SCPS_ERR_INVALID_ARG, "NULL descriptor or output pointer");
    *out = nullptr;
    if (d->model != SCPS_MODEL_CHAIN && !is_2d(d->model))
        return fail(SCPS_ERR_INVALID_ARG, "unknown model %d", d->model);
    if (d->n_replicas <= 0) return fail(SCPS_ERR_INVALID_ARG, "n_replicas must be > 0");
    if (!d->x0) return fail(SCPS_ERR_INVALID_ARG, "x0 is NULL");
    if (!(d->dt > 0.0) || !(d->gamma > 0.0) || !(d->kT >= 0.0))
        return fail(SCPS_ERR_INVALID_ARG, "need dt > 0, gamma > 0, kT >= 0");
    if (d->save_interval < 0 || (d->save_interval > 0 && d->max_frames <= 0))
        return fail(SCPS_ERR_INVALID_ARG, "save_interval > 0 needs max_frames > 0");
    if (d->exec != SCPS_EXEC_RESIDENT && d->exec != SCPS_EXEC_PLAIN)
        return fail(SCPS_ERR_INVALID_ARG, "unknown exec form %d", d->exec);
    if (d->cluster_size < 0 || d->cluster_size > 2)
        return fail(SCPS_ERR_UNSUPPORTED, "cluster_size %d not supported (0, 1 or 2)", d->cluster_size);
    if (d->threads != 0 && (d->threads < 128 || d->threads > 1024 || d->threads % 32))
        return fail(SCPS_ERR_INVALID_ARG, "threads must be 0 or a multiple of 32 in [128, 1024]");
    if (d->cluster_size == 2 && d->threads > kMaxThreadsPair)
        return fail(SCPS_ERR_INVALID_ARG, "a 2-CTA cluster takes at most %d threads per CTA",
                    kMaxThreadsPair);
    scps_system* s = new scps_system();
    s->d = *d;
    s->d.topologies = nullptr;
    s->d.replica_topology = nullptr;
    s->d.replica_id = nullptr;
    s->d.x0 = nullptr;
    s->d.v0 = nullptr;
    s->model = d->model;
    cudaGetDevice(&s->device);
    const int R = d->n_replicas;
    s->rep_id.resize(R);
    for (int r = 0; r < R; ++r) s->rep_id[r] = d->replica_id ? (uint32_t)d->replica_id[r] : (uint32_t)r;
    s->host_step.assign(R, 0);
    auto bail = [&](int rc) {
        scps_destroy_system(s);
        return rc;
    };
    if (d->model == SCPS_MODEL_CHAIN) {
        if (d->n_topologies <= 0 || !d->topologies || !d->replica_topology)
            return bail(fail(SCPS_ERR_INVALID_ARG, "chain model needs topologies and replica_topology"));
        if (!(d->cutoff > 0.0)) return bail(fail(SCPS_ERR_INVALID_ARG, "cutoff must be > 0"));
        s->is_box = d->box != 0.0;
        if (s->is_box) {
            const double skin = d->skin > 0.0 ? d->skin : 0.15;
            if (!(d->box > 2.0 * (d->cutoff + skin)))
                return bail(fail(SCPS_ERR_INVALID_ARG, "box %.3f nm is too small for cutoff + skin",
                                 d->box));
            if (d->n_topologies != 1)
                return bail(fail(SCPS_ERR_UNSUPPORTED, "the periodic box takes one topology"));
            if (d->exec != SCPS_EXEC_RESIDENT)
                return bail(fail(SCPS_ERR_UNSUPPORTED, "the periodic box has one execution form"));
        }
        if (d->elec < SCPS_ELEC_NONE || d->elec > SCPS_ELEC_PLAIN)
            return bail(fail(SCPS_ERR_INVALID_ARG, "unknown electrostatics %d", d->elec));
        if (d->elec == SCPS_ELEC_DDIEL && !(d->k_dd > 0.0))
            return bail(fail(SCPS_ERR_INVALID_ARG, "k_dd must be > 0"));
        if (d->integrator != SCPS_INT_BAOAB)
            return bail(fail(SCPS_ERR_UNSUPPORTED, "the chain model integrates with BAOAB"));
        s->topos.resize(d->n_topologies);
        for (int t = 0; t < d->n_topologies; ++t) {
            int rc = validate_topology(d->topologies[t], t, s->is_box ? kMaxBoxAtoms : kMaxChainAtoms);
            if (rc) return bail(rc);
            rc = build_topology(s, d->topologies[t], s->topos[t]);
            if (rc) return bail(rc);
            s->max_atoms = std::max(s->max_atoms, s->topos[t].n);
        }
        s->rep_topo.resize(R);
        for (int r = 0; r < R; ++r) {
            const int t = d->replica_topology[r];
            if (t < 0 || t >= d->n_topologies)
                return bail(fail(SCPS_ERR_INVALID_ARG, "replica %d: topology %d out of range", r, t));
            s->rep_topo[r] = t;
        }
    } else {
        if (d->integrator != SCPS_INT_EM)
            return bail(fail(SCPS_ERR_UNSUPPORTED, "the toy model integrates with Euler-Maruyama"));
        s->max_atoms = 1;
    }
    // packed addressing
    s->atom_off.resize(R);
    s->frame_off.resize(R);
    long long off = 0, foff = 0;
    for (int r = 0; r < R; ++r) {
        const int n = atoms_per_replica(s, r);
        s->atom_off[r] = (int)off;
        s->frame_off[r] = foff;
        off += n;
        foff += (long long)std::max(d->max_frames, 0) * n;
    }
    s->n_atoms_total = off;
    s->n_frame_atoms = foff;
    const int mf = std::max(d->max_frames, 1);
    const int dims = is_2d(d->model) ? 2 : 3;
    StateDev& st = s->st;
    int rc = 0;
#define ALLOC(p, n)                                          \
    do {                                                     \
        cudaError_t e_ = s->alloc(&(p), (size_t)(n));        \
        if (e_ != cudaSuccess)                               \
            return bail(fail(SCPS_ERR_CUDA, "cudaMalloc: %s", cudaGetErrorString(e_))); \
    } while (0)
    const int Rs = R + (s->is_box ? 1 : 0);  // the box keeps one more slot for evaluations
    ALLOC(st.zm, Rs);
    ALLOC(st.z, Rs);
    ALLOC(st.step, Rs);
    ALLOC(st.T, Rs);
    ALLOC(st.status, Rs);
    ALLOC(st.n_saved, Rs);
    ALLOC(st.fz, (size_t)R * mf);
    ALLOC(st.fzm, (size_t)R * mf);
    ALLOC(st.fe, (size_t)R * mf);
    ALLOC(st.fT, (size_t)R * mf);
    ALLOC(st.frames, (size_t)std::max(foff, 1ll) * dims);
    ALLOC(s->d_rep_ids, R);
    if (d->model == SCPS_MODEL_CHAIN) {
        ALLOC(st.x, off);
        ALLOC(st.v, off);
        ALLOC(st.sm, R);
        ALLOC(st.wm, R);
        ALLOC(s->d_topos, s->topos.size());
        ALLOC(s->d_reps, R);
        ALLOC(s->plain_f, (size_t)6 * s->max_atoms + 16384 + 64);
        ALLOC(s->plain_d, 8);
        ALLOC(st.pair_slots, R);
        ALLOC(st.list_builds, R);
    } else {
        ALLOC(st.xy, R);
        ALLOC(st.sm, R);
        ALLOC(st.wm, R);
    }
#undef ALLOC
    {
        std::vector<double> inf(R, std::numeric_limits<double>::infinity());
        cudaMemcpy(st.zm, inf.data(), sizeof(double) * R, cudaMemcpyHostToDevice);
        cudaMemcpy(s->d_rep_ids, s->rep_id.data(), sizeof(uint32_t) * R, cudaMemcpyHostToDevice);
    }
    if (d->model == SCPS_MODEL_CHAIN) {
        s->nta = ((s->max_atoms + kTile - 1) / kTile) * kTile;
        if (!s->is_box && d->exec == SCPS_EXEC_RESIDENT) {  // pair-list slabs
            s->list_slab = list_slab_bytes(s->nta);
            cudaError_t e_ = s->alloc(&s->d_lists, (size_t)R * (size_t)s->list_slab);
            if (e_ != cudaSuccess)
                return bail(fail(SCPS_ERR_CUDA, "cudaMalloc of the pair lists: %s", cudaGetErrorString(e_)));
        }
        std::vector<RepDev> reps(R);
        for (int r = 0; r < R; ++r)
            reps[r] = RepDev{s->rep_topo[r], s->atom_off[r], s->frame_off[r], s->rep_id[r], r,
                             (long long)r * s->list_slab};
        if (cudaMemcpy(s->d_reps, reps.data(), sizeof(RepDev) * R, cudaMemcpyHostToDevice) != cudaSuccess)
            return bail(fail(SCPS_ERR_CUDA, "upload of the replica table failed"));
        rc = sync_topos(s);
        if (rc) return bail(rc);
        int n_sm = 0;
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, s->device);
        // a 2-CTA cluster per replica when the replicas alone leave SMs idle
        s->cluster = d->cluster_size
                         ? d->cluster_size
                         : (2 * R <= n_sm && d->threads <= kMaxThreadsPair ? 2 : 1);
        const bool one_cta_per_sm = (long long)R * s->cluster <= n_sm;
        s->threads = d->threads ? d->threads : (one_cta_per_sm ? 1024 : auto_threads(s->nta));
        if (s->cluster == 2 && !d->threads) s->threads = std::min(s->threads, kMaxThreadsPair);
        s->steps_per_graph = d->steps_per_graph > 0 ? d->steps_per_graph : 1000;
        if (!s->is_box && d->exec == SCPS_EXEC_RESIDENT) {
            const size_t smem = resident_smem_bytes(s->nta);
            if (smem > resident_smem_limit())
                return bail(fail(SCPS_ERR_UNSUPPORTED,
                                 "%d atoms need %zu B of shared memory per CTA, above the limit; "
                                 "use the plain execution form", s->max_atoms, smem));
            rc = set_groups(s, 0, s->cluster, s->threads);
            if (rc) return bail(rc);
        }
    }
    if (s->is_box) {
        const scps_topology_desc& t = d->topologies[0];
        int nch = 0;  // bonded atoms come first: the chain is atoms [0, nch)
        for (int b = 0; b < 2 * t.n_bonds; ++b) nch = std::max(nch, t.bonds[b] + 1);
        for (int a = 0; a < 3 * t.n_angles; ++a) nch = std::max(nch, t.angles[a] + 1);
        for (int e = 0; e < 2 * t.n_excl; ++e) nch = std::max(nch, t.excl[e] + 1);
        BoxDev& B = s->box;
        B.n_atoms = t.n_atoms;
        B.n_chain = std::max(nch, 1);
        // columns about as wide as a cube holding 32 atoms; every column starts
        // a tile, so ncol^2 tiles more than ceil(n / 32) always suffice
        const double cube = std::cbrt(32.0 * d->box * d->box * d->box / t.n_atoms);
        B.ncol = std::max(1, std::min(16, (int)std::lround(d->box / cube)));
        B.nz = 8192 / (B.ncol * B.ncol);
        B.nt = (t.n_atoms + kTile - 1) / kTile + B.ncol * B.ncol;
        B.np = B.nt * kTile;
        // pair-list capacity per 8-slot cluster: its own slots and the atoms within r_c +
        // 0.75 nm of its centre at the mean density (the union of the cluster's atoms' list
        // spheres for skins up to the tuner's 0.2 nm, with room for fluctuations). A list
        // holds only later clusters, but for the clusters of the first columns in slot
        // order that is nearly the whole sphere.
        {
            const double rho = t.n_atoms / (d->box * d->box * d->box);
            const double rr = d->cutoff + 0.75;
            const double full = rho * 4.18879020478639 * rr * rr * rr;
            B.max_ent = std::min(1 << 14, 8 + 8 * (int)std::ceil(full / 8.0));
        }
        B.rebuild_every = d->rebuild_every > 0 ? d->rebuild_every : 20;
        B.L = (float)d->box;
        B.invL = (float)(1.0 / d->box);
        const double skin = d->skin > 0.0 ? d->skin : 0.15;
        B.rlist2 = (float)((d->cutoff + skin) * (d->cutoff + skin));
        B.skin2_quarter = (float)(0.25 * skin * skin);
        const size_t np = (size_t)Rs * B.np;
#define BALLOC(p, n)                                                                        \
    do {                                                                                    \
        cudaError_t e_ = s->alloc(&(p), (size_t)(n));                                       \
        if (e_ != cudaSuccess)                                                              \
            return bail(fail(SCPS_ERR_CUDA, "cudaMalloc: %s", cudaGetErrorString(e_)));     \
    } while (0)
        BALLOC(B.pos, np);
        BALLOC(B.vel, np);
        BALLOC(B.par, np);
        BALLOC(B.id, np);
        BALLOC(B.id2, np);
        BALLOC(B.facc, 3 * np);
        BALLOC(B.epair, Rs);
        if (cudaMemset(B.facc, 0, sizeof(long long) * 3 * np) != cudaSuccess ||
            cudaMemset(B.epair, 0, sizeof(long long) * Rs) != cudaSuccess)
            return bail(fail(SCPS_ERR_CUDA, "cudaMemset failed"));
        BALLOC(B.pos2, np);
        BALLOC(B.vel2, np);
        BALLOC(B.key, np);
        BALLOC(B.hist, (size_t)Rs * 8192);
        BALLOC(B.colinfo, (size_t)Rs * 2 * 257);
        BALLOC(B.pos_ref, np);
        BALLOC(B.slot_of, (size_t)Rs * B.n_atoms);
        BALLOC(B.clo, (size_t)Rs * 4 * B.nt);  // per 8-slot cluster
        BALLOC(B.chi, (size_t)Rs * 4 * B.nt);
        BALLOC(B.ent, (size_t)Rs * 4 * B.nt * B.max_ent);
        BALLOC(B.nent, (size_t)Rs * 4 * B.nt);
        BALLOC(B.cflag, (size_t)Rs * 4 * B.nt);
        BALLOC(B.need, Rs);
        BALLOC(B.since, Rs);
        BALLOC(B.nbuild, Rs);
        BALLOC(B.nevent, 1);
        BALLOC(B.maxd2, Rs);
        BALLOC(B.fch, (size_t)Rs * B.n_chain);
        BALLOC(B.eb, Rs);
#undef BALLOC
        if (box_chain_smem(B.n_chain, 0) > box_chain_smem_limit())
            return bail(fail(SCPS_ERR_UNSUPPORTED, "chain of %d atoms is too large for one CTA",
                             B.n_chain));
        if (box_prepare(B, 0) != cudaSuccess) return bail(fail(SCPS_ERR_CUDA, "box set-up failed"));
    }
    rc = scps_set_state(s, d->x0, d->v0, nullptr, nullptr, nullptr);
    if (rc) return bail(rc);
    if (cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
        return bail(fail(SCPS_ERR_CUDA, "cudaStreamCreate failed"));
    if (s->is_box && (cudaStreamCreateWithFlags(&s->box_graphs.cap, cudaStreamNonBlocking) != cudaSuccess ||
                      cudaStreamCreateWithFlags(&s->box_graphs.cap2, cudaStreamNonBlocking) != cudaSuccess))
        return bail(fail(SCPS_ERR_CUDA, "cudaStreamCreate failed"));
    // run parameters shared by every launch
    RunParams& P = s->base;
    P.n_replicas = R;
    P.dt = (float)d->dt;
    P.half_dt = (float)(0.5 * d->dt);
    P.c1 = (float)std::exp(-d->gamma * d->dt);
    P.gamma = d->gamma;
    P.key0 = (uint32_t)(d->seed & 0xffffffffull);
    P.key1 = (uint32_t)(d->seed >> 32);
    P.save_interval = d->save_interval;
    P.max_frames = mf;
    P.bias = 0;
    P.k_R = 0.0;
    P.toy_dt_over_gamma = d->dt / d->gamma;
    P.toy_sd = std::sqrt(2.0 * d->kT * d->dt / d->gamma);
    P.toy_x_ref = 1.0;
    P.toy_model = d->model == SCPS_MODEL_FUNNEL2D ? 1 : 0;
    const double rcut = d->cutoff > 0.0 ? d->cutoff : 1.0;
    P.pc.rc = (float)rcut;
    P.pc.rc2 = (float)(rcut * rcut);
    P.pc.inv_rc = (float)(1.0 / rcut);
    P.pc.inv_rc2 = (float)(1.0 / (rcut * rcut));
    P.pc.inv_rc3 = (float)(1.0 / (rcut * rcut * rcut));
    const double krf = (d->eps_rf - 1.0) / ((2.0 * d->eps_rf + 1.0) * rcut * rcut * rcut);
    P.pc.krf = (float)krf;
    P.pc.crf = (float)(1.0 / rcut + krf * rcut * rcut);
    // the 2^-13 pair terms of one item (8 per accumulator) stay below 2^31 while
    // |s| r_c 2^13 8 < 2^31; larger |s| take the exact slow path
    P.pc.s_lim = (float)(32000.0 / rcut);
    // pair list of the resident chain kernels (the periodic box keeps its own)
    const double skin = d->skin > 0.0 ? d->skin : (s->is_box ? 0.15 : kDefaultChainSkin);
    P.list_base = s->d_lists;
    set_skin(s, skin);
    P.rebuild_every = s->is_box ? 0 : std::max(d->rebuild_every, 0);
    *out = s;
    return SCPS_OK;
}

int scps_destroy_system(scps_system* s) {
    TraceRange trace_("scps_destroy_system");
    if (!s) return SCPS_OK;
    drop_graphs(s);
    if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
    if (s->box_graphs.cap) cudaStreamDestroy(s->box_graphs.cap);
    if (s->box_graphs.cap2) cudaStreamDestroy(s->box_graphs.cap2);
    s->drop_bias_tables();
    for (auto st : s->fork_streams) cudaStreamDestroy(st);
    for (auto ev : s->fork_events) cudaEventDestroy(ev);
    for (void* p : s->allocs) cudaFree(p);
    if (s->d_eval_lists) cudaFree(s->d_eval_lists);
    delete s;
    return SCPS_OK;
}

int scps_set_bias(scps_system* s, const scps_bias_desc* b) {
    TraceRange trace_("scps_set_bias");
    if (!s || !b) return fail(SCPS_ERR_INVALID_ARG, "NULL system or bias");
    RunParams& P = s->base;
    // the previous bias goes first (its tables are freed once no enqueued work can read
    // them); a call that fails below leaves the system without a bias
    SCPS_CU(cudaDeviceSynchronize());
    drop_graphs(s);
    s->drop_bias_tables();
    P.bias = 0;
    P.tube_k = 0;
    for (auto& t : s->topos) {
        t.dev.n_contacts = 0;
        t.dev.con_ij = nullptr;
        t.dev.con_C0 = nullptr;
        t.dev.con_off = nullptr;
        t.dev.con_nbr = nullptr;
        t.dev.tube_A = nullptr;
        t.ncon = 0;
    }
    if (s->model == SCPS_MODEL_CHAIN) {
        int rc0 = sync_topos(s);
        if (rc0) return rc0;
    }
    if (b->kind == SCPS_BIAS_NONE) {
        P.bias = 0;
    } else if (b->kind == SCPS_BIAS_RMD_TOY || b->kind == SCPS_BIAS_RMD_RADIAL) {
        if (!is_2d(s->model)) return fail(SCPS_ERR_INVALID_ARG, "toy bias on a chain system");
        P.bias = b->kind == SCPS_BIAS_RMD_TOY ? 2 : 3;
        P.toy_x_ref = b->toy_x_ref;
    } else if (b->kind == SCPS_BIAS_TUBE && is_2d(s->model)) {
        if (b->n_ref < 1 || b->n_ref > 1000000 || !b->ref || !b->ref_time)
            return fail(SCPS_ERR_INVALID_ARG, "tube bias needs 1 <= n_ref <= 1e6, ref and ref_time");
        if (!(b->lambda > 0.0) || !(b->t_path > 0.0) || !(b->k_s >= 0.0) || !(b->k_w >= 0.0))
            return fail(SCPS_ERR_INVALID_ARG, "tube bias needs lambda > 0, t_path > 0, k_s, k_w >= 0");
        std::vector<double2> ref(b->n_ref);
        std::vector<double> tm(b->ref_time, b->ref_time + b->n_ref);
        for (int k = 0; k < b->n_ref; ++k) {
            ref[k] = make_double2(b->ref[2 * k], b->ref[2 * k + 1]);
            if (!std::isfinite(ref[k].x) || !std::isfinite(ref[k].y) || !std::isfinite(tm[k]))
                return fail(SCPS_ERR_NONFINITE, "non-finite reference point %d", k);
        }
        double2* d_ref = nullptr;
        double* d_tm = nullptr;
        SCPS_CU(s->bias_upload(&d_ref, ref));
        SCPS_CU(s->bias_upload(&d_tm, tm));
        P.bias = 4;
        P.tube_k = b->n_ref;
        P.tube_ref = d_ref;
        P.tube_time = d_tm;
        P.tube_lambda = b->lambda;
        P.tube_ks = b->k_s;
        P.tube_kw = b->k_w;
        P.tube_t = b->t_path;
    } else if (b->kind == SCPS_BIAS_RMD_CONTACTS || b->kind == SCPS_BIAS_TUBE) {
        if (s->model != SCPS_MODEL_CHAIN) return fail(SCPS_ERR_INVALID_ARG, "contact bias needs the chain model");
        if (!(b->r0 > 0.0)) return fail(SCPS_ERR_INVALID_ARG, "r0 must be > 0");
        if (!b->n_pairs || !b->pairs || !b->x_native)
            return fail(SCPS_ERR_INVALID_ARG, "contact bias needs n_pairs, pairs and x_native");
        const bool tube = b->kind == SCPS_BIAS_TUBE;
        if (tube) {
            if (s->is_box || s->d.exec != SCPS_EXEC_RESIDENT)
                return fail(SCPS_ERR_UNSUPPORTED, "the contact-map tube bias runs in the resident form of chains");
            if (b->n_ref < 1 || b->n_ref > kMaxTubeK || !b->ref_maps || !b->ref_time)
                return fail(SCPS_ERR_INVALID_ARG, "tube bias needs 1 <= n_ref <= %d, ref_maps and ref_time",
                            kMaxTubeK);
            if (!(b->lambda > 0.0) || !(b->t_path > 0.0) || !(b->k_s >= 0.0) || !(b->k_w >= 0.0))
                return fail(SCPS_ERR_INVALID_ARG, "tube bias needs lambda > 0, t_path > 0, k_s, k_w >= 0");
        }
        const double inv_r0sq = 1.0 / (b->r0 * b->r0);
        int ncon_max = 0;
        for (size_t t = 0; t < s->topos.size(); ++t) {
            const int nc = b->n_pairs[t], n = s->topos[t].n;
            if (nc < 0) return fail(SCPS_ERR_INVALID_ARG, "topology %zu: negative pair count", t);
            if (nc > 0 && (!b->pairs[t] || !b->x_native[t]))
                return fail(SCPS_ERR_INVALID_ARG, "topology %zu: NULL pairs or x_native", t);
            std::vector<int2> pairs(nc);
            for (int c = 0; c < nc; ++c) {
                const int i = b->pairs[t][2 * c], j = b->pairs[t][2 * c + 1];
                if (i < 0 || j < 0 || i >= n || j >= n || i == j)
                    return fail(SCPS_ERR_INVALID_ARG, "topology %zu: contact %d has bad atoms", t, c);
                pairs[c] = make_int2(i, j);
            }
            std::vector<double> xn(nc > 0 ? (size_t)3 * n : 0);
            if (nc > 0) std::memcpy(xn.data(), b->x_native[t], sizeof(double) * 3 * n);
            // per-atom adjacency of the contact list: (contact index, partner atom)
            std::vector<int> off(n + 1, 0);
            for (int c = 0; c < nc; ++c) {
                off[pairs[c].x + 1]++;
                off[pairs[c].y + 1]++;
            }
            for (int i = 0; i < n; ++i) off[i + 1] += off[i];
            std::vector<int> fill(off.begin(), off.end() - 1);
            std::vector<int2> nbr((size_t)2 * nc);
            for (int c = 0; c < nc; ++c) {
                nbr[fill[pairs[c].x]++] = make_int2(c, pairs[c].y);
                nbr[fill[pairs[c].y]++] = make_int2(c, pairs[c].x);
            }
            int2* d_pairs;
            float2* d_c0;
            double* d_xn;
            int* d_off;
            int2* d_nbr;
            SCPS_CU(s->bias_upload(&d_pairs, pairs));
            SCPS_CU(s->bias_upload(&d_c0, std::vector<float2>(std::max(nc, 1))));
            SCPS_CU(s->bias_upload(&d_off, off));
            SCPS_CU(s->bias_upload(&d_nbr, nbr));
            SCPS_CU(cudaMalloc(&d_xn, sizeof(double) * std::max<size_t>(xn.size(), 1)));
            if (!xn.empty()) {
                cudaError_t ex = cudaMemcpy(d_xn, xn.data(), sizeof(double) * xn.size(), cudaMemcpyHostToDevice);
                if (ex != cudaSuccess) {
                    cudaFree(d_xn);
                    return fail(SCPS_ERR_CUDA, "upload of x_native failed: %s", cudaGetErrorString(ex));
                }
            }
            cudaError_t em = launch_native_map(nc, d_pairs, d_xn, inv_r0sq, d_c0, 0);
            if (em == cudaSuccess) em = cudaDeviceSynchronize();
            cudaFree(d_xn);  // only C0 = C(X_N) is kept
            SCPS_CU(em);
            if (tube) {  // reference maps, stored [item of kTubeItem contacts][slice][contact
                         // of the item], zero past the last contact; N0 = sum C0^2 (Eq. sX)
                if (nc > 0 && !b->ref_maps[t])
                    return fail(SCPS_ERR_INVALID_ARG, "topology %zu: NULL reference maps", t);
                const int K = b->n_ref;
                const size_t n_it = (size_t)std::max((nc + kTubeItem - 1) / kTubeItem, 1);
                std::vector<float> A(n_it * K * kTubeItem, 0.f);
                double n0 = 0.0;
                for (int c = 0; c < nc; ++c) {
                    double d2 = 0.0;
                    for (int k = 0; k < 3; ++k) {
                        const double dd = xn[3 * pairs[c].y + k] - xn[3 * pairs[c].x + k];
                        d2 += dd * dd;
                    }
                    const double u = d2 * inv_r0sq, num = 1.0 + u + u * u;
                    const double c0 = num / (num + u * u * u + u * u * u * u);
                    n0 += c0 * c0;
                    for (int k = 0; k < K; ++k) {
                        const double a = b->ref_maps[t][(size_t)k * nc + c];
                        if (!std::isfinite(a))
                            return fail(SCPS_ERR_NONFINITE, "topology %zu: non-finite reference map", t);
                        A[((size_t)(c / kTubeItem) * K + k) * kTubeItem + c % kTubeItem] = (float)a;
                    }
                }
                float* d_A;
                SCPS_CU(s->bias_upload(&d_A, A));
                s->topos[t].dev.tube_A = d_A;
                s->topos[t].dev.tube_inv_n0 = n0 > 0.0 ? (float)(1.0 / n0) : 0.f;
            }
            s->topos[t].dev.n_contacts = nc;
            s->topos[t].dev.con_ij = d_pairs;
            s->topos[t].dev.con_C0 = d_c0;
            s->topos[t].dev.con_off = d_off;
            s->topos[t].dev.con_nbr = d_nbr;
            s->topos[t].ncon = nc;
            ncon_max = std::max(ncon_max, nc);
        }
        if (s->is_box) {
            for (int c = 0; c < b->n_pairs[0]; ++c)
                if (b->pairs[0][2 * c] >= s->box.n_chain || b->pairs[0][2 * c + 1] >= s->box.n_chain)
                    return fail(SCPS_ERR_INVALID_ARG, "contact %d is not between chain atoms", c);
            const size_t smem = sizeof(float4) * s->box.n_chain + sizeof(long long) * 3 * s->box.n_chain +
                                sizeof(float) * ncon_max;
            if (smem > box_chain_smem_limit())
                return fail(SCPS_ERR_UNSUPPORTED, "chain of %d atoms and %d contacts is too large",
                            s->box.n_chain, ncon_max);
            SCPS_CU(box_prepare(s->box, ncon_max));
        } else {
            const size_t smem = resident_smem_bytes(s->nta);
            if (s->d.exec == SCPS_EXEC_RESIDENT && smem > resident_smem_limit())
                return fail(SCPS_ERR_UNSUPPORTED, "shared memory %zu B exceeds the per-CTA limit", smem);
        }
        if (s->d.exec == SCPS_EXEC_PLAIN && ncon_max > 16384)
            return fail(SCPS_ERR_UNSUPPORTED, "plain form supports up to 16384 contacts");
        s->ncon_max = ncon_max;
        int rc = sync_topos(s);
        if (rc) return rc;
        P.bias = 1;
        s->inv_r0sq = inv_r0sq;
        P.inv_r0sq = (float)inv_r0sq;
        const float hi = (float)inv_r0sq;
        P.inv_r0sq_ff = ff{hi, (float)(inv_r0sq - (double)hi)};
        if (tube) {
            std::vector<double> tm(b->ref_time, b->ref_time + b->n_ref);
            for (double v : tm)
                if (!std::isfinite(v)) return fail(SCPS_ERR_NONFINITE, "non-finite reference time");
            double* d_tm = nullptr;
            SCPS_CU(s->bias_upload(&d_tm, tm));
            P.bias = 5;
            P.tube_k = b->n_ref;
            P.tube_time = d_tm;
            P.tube_lambda = b->lambda;
            P.tube_ks = b->k_s;
            P.tube_kw = b->k_w;
            P.tube_t = b->t_path;
        }
    } else {
        return fail(SCPS_ERR_INVALID_ARG, "unknown bias kind %d", b->kind);
    }
    P.k_R = b->k_R;
    s->bias_kind = b->kind;
    const int R = s->d.n_replicas;
    std::vector<double> zm(R, b->zm_init == SCPS_ZM_VALUE ? b->zm_value
                                                          : std::numeric_limits<double>::infinity());
    std::vector<double> zero(R, 0.0);
    SCPS_CU(cudaMemcpy(s->st.zm, zm.data(), sizeof(double) * R, cudaMemcpyHostToDevice));
    SCPS_CU(cudaMemcpy(s->st.T, zero.data(), sizeof(double) * R, cudaMemcpyHostToDevice));
    if (s->st.sm) {  // s_m and w_m of the tube bias follow the same initial rule as z_m
        SCPS_CU(cudaMemcpy(s->st.sm, zm.data(), sizeof(double) * R, cudaMemcpyHostToDevice));
        SCPS_CU(cudaMemcpy(s->st.wm, zm.data(), sizeof(double) * R, cudaMemcpyHostToDevice));
    }
    drop_graphs(s);
    return SCPS_OK;
}

int scps_step_replicas(scps_system* s, int64_t n_steps, void* stream) {
    TraceRange trace_("scps_step_replicas");
    if (!s) return fail(SCPS_ERR_INVALID_ARG, "NULL system");
    if (n_steps < 0) return fail(SCPS_ERR_INVALID_ARG, "n_steps must be >= 0");
    if (n_steps == 0) return SCPS_OK;
    cudaStream_t cs = (cudaStream_t)stream;
    const int R = s->d.n_replicas;
    for (int r = 0; r < R; ++r)
        if (s->host_step[r] + n_steps > (long long)UINT32_MAX)
            return fail(SCPS_ERR_INVALID_ARG, "step counter would pass 2^32 (noise counter word)");
    RunParams P = s->base;
    long long launches = 0;
    if (is_2d(s->model)) {
        P.n_steps = n_steps;
        SCPS_CU(launch_toy(s->st, P, s->d_rep_ids, cs));
        launches = 1;
    } else if (s->is_box) {
        for (int r = 1; r < R; ++r)
            if (s->host_step[r] != s->host_step[0])
                return fail(SCPS_ERR_STATE, "periodic-box replicas must share one step counter");
        const long long frame_atoms = (long long)std::max(s->d.max_frames, 1) * s->box.n_atoms;
        SCPS_CU(cudaMemsetAsync(s->box.nbuild, 0, sizeof(int) * (size_t)(R + 1), cs));
        SCPS_CU(cudaMemsetAsync(s->box.nevent, 0, sizeof(int), cs));
        SCPS_CU(box_run(s->box, s->d_topos, s->st, P, s->d_rep_ids, R, s->d.elec, s->ncon_max,
                        s->host_step[0], n_steps, frame_atoms, &s->box_graphs, cs));
        // the evaluation that opens the call (decide, hist clear, 7 rebuild kernels that
        // return at once unless a rebuild is forced, pairs, chain) and its A half step; per
        // step one graph of 5 kernels (step counter, decide, pairs, chain, integrate; 2 more
        // on save steps) plus 8 inside its conditional node on the steps that rebuild (added
        // by scps_get_info, which reads their count)
        launches = 12 + 5 * n_steps;
        s->last_launch_steps = n_steps;
    } else if (s->d.exec == SCPS_EXEC_PLAIN) {
        P.n_steps = n_steps;
        std::vector<RepDev> reps(R);
        for (int r = 0; r < R; ++r) {
            const RepDev rep{s->rep_topo[r], s->atom_off[r], s->frame_off[r], s->rep_id[r], r};
            SCPS_CU(plain_run_replica(s->d.elec, s->topos[s->rep_topo[r]].dev, s->st, r, rep, P,
                                      s->plain_f, s->plain_d, s->host_step[r], cs));
        }
        SCPS_CU(launch_add_steps(s->st.step, R, n_steps, cs));
        launches = -1;  // many; not tracked
    } else {
        const long long chunk = s->steps_per_graph;
        const long long full = n_steps / chunk, rem = n_steps % chunk;
        if (full > 0) {
            auto it = s->graphs.find(chunk);
            if (it == s->graphs.end()) {
                RunParams Pc = P;
                Pc.n_steps = chunk;
                cudaGraph_t g;
                SCPS_CU(cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal));
                cudaError_t le = launch_groups(s, Pc, chunk, s->cap_stream);
                cudaError_t ce = cudaStreamEndCapture(s->cap_stream, &g);
                if (le != cudaSuccess || ce != cudaSuccess)
                    return fail(SCPS_ERR_CUDA, "graph capture failed: %s",
                                cudaGetErrorString(le != cudaSuccess ? le : ce));
                cudaGraphExec_t ge;
                SCPS_CU(cudaGraphInstantiate(&ge, g, 0));
                s->graph_defs.push_back(g);
                it = s->graphs.emplace(chunk, ge).first;
            }
            for (long long k = 0; k < full; ++k) SCPS_CU(cudaGraphLaunch(it->second, cs));
        }
        if (rem > 0) {
            P.n_steps = rem;
            SCPS_CU(launch_groups(s, P, rem, cs));
        }
        launches = (full + (rem > 0)) * (long long)s->groups.size();
        s->last_launch_steps = rem > 0 ? rem : chunk;
    }
    for (int r = 0; r < R; ++r) s->host_step[r] += n_steps;
    s->info.graph_nodes_last_call = launches;
    return SCPS_OK;
}

int scps_energy_forces(scps_system* s, int32_t topo, int64_t n_frames, const float* X, double* U,
                       float* F, double* z, void* stream) {
    TraceRange trace_("scps_energy_forces");
    if (!s) return fail(SCPS_ERR_INVALID_ARG, "NULL system");
    if (s->model != SCPS_MODEL_CHAIN) return fail(SCPS_ERR_UNSUPPORTED, "chain model only");
    if (topo < 0 || topo >= (int)s->topos.size()) return fail(SCPS_ERR_INVALID_ARG, "bad topology %d", topo);
    if (n_frames < 0 || n_frames > 2147483647ll) return fail(SCPS_ERR_INVALID_ARG, "bad n_frames");
    if (n_frames == 0) return SCPS_OK;
    if (!X || !U) return fail(SCPS_ERR_INVALID_ARG, "X and U are required");
    if (z && s->base.bias != 1 && s->base.bias != 5)
        return fail(SCPS_ERR_STATE, "z needs the contact list of a contact or tube bias (scps_set_bias)");
    if (s->is_box) {  // frame by frame in the evaluation slot of the box
        RunParams P = s->base;
        if (!z) P.bias = 0;
        const int n = s->box.n_atoms;
        for (long long f = 0; f < n_frames; ++f)
            SCPS_CU(box_energy_forces(s->box, s->d_topos, s->st, P, s->d.n_replicas, s->d.elec,
                                      s->ncon_max, X + f * n * 3, U + f, F ? F + f * n * 3 : nullptr,
                                      z ? z + f : nullptr, (cudaStream_t)stream));
        return SCPS_OK;
    }
    const TopoHost& th = s->topos[topo];
    const int nta = ((th.n + kTile - 1) / kTile) * kTile;
    RunParams P = s->base;
    if (!z) P.bias = 0;
    P.rlist2 = P.pc.rc2;  // one list per frame: no skin needed
    // list slabs: one per frame cluster of a launch (grown on demand; the previous
    // buffer is freed once no enqueued work can still read it)
    const long long per_launch = std::min<long long>(n_frames, kEvalFramesPerLaunch);
    const long long slab = list_slab_bytes(nta);
    if (per_launch > s->eval_frames_cap || slab > s->eval_slab) {
        const long long cap = std::max(per_launch, s->eval_frames_cap);
        const long long sl = std::max(slab, s->eval_slab);
        SCPS_CU(cudaDeviceSynchronize());
        if (s->d_eval_lists) {
            cudaFree(s->d_eval_lists);
            s->bytes -= (size_t)(s->eval_frames_cap * s->eval_slab);
            s->d_eval_lists = nullptr;
        }
        s->eval_frames_cap = 0;
        s->eval_slab = 0;
        SCPS_CU(cudaMalloc(&s->d_eval_lists, (size_t)(cap * sl)));
        s->eval_frames_cap = cap;
        s->eval_slab = sl;
        s->bytes += (size_t)(cap * sl);
    }
    P.list_base = s->d_eval_lists;
    P.list_slab = s->eval_slab;
    // few frames (a checkpoint segment): a 2-CTA cluster per frame, 1024 threads per CTA,
    // so that the frames spread over the SMs; many frames: one CTA each
    int n_sm = 0;
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, s->device);
    const int n3 = 3 * th.n;
    for (long long f0 = 0; f0 < n_frames; f0 += per_launch) {
        const long long nf = std::min(per_launch, n_frames - f0);
        const int cl = 2 * nf <= n_sm ? 2 : 1;
        const int threads = nf * cl <= n_sm ? 1024 : auto_threads(nta);
        SCPS_CU(launch_eval(s->d.elec, s->d_topos + topo, P, X + f0 * n3, U + f0,
                            F ? F + f0 * n3 : nullptr, z ? z + f0 : nullptr, nf, nta, threads, cl,
                            (cudaStream_t)stream));
    }
    return SCPS_OK;
}

int scps_hvp(scps_system* s, int32_t topo, int64_t n_frames, const float* X, const float* V,
             float* HV, void* stream) {
    TraceRange trace_("scps_hvp");
    if (!s) return fail(SCPS_ERR_INVALID_ARG, "NULL system");
    if (s->model != SCPS_MODEL_CHAIN) return fail(SCPS_ERR_UNSUPPORTED, "chain model only");
    if (s->is_box)  // these kernels take every pair once, with no periodic images
        return fail(SCPS_ERR_UNSUPPORTED, "Hessian-vector products cover open-boundary chains");
    if (topo < 0 || topo >= (int)s->topos.size()) return fail(SCPS_ERR_INVALID_ARG, "bad topology %d", topo);
    if (n_frames < 0 || n_frames > 2147483647ll) return fail(SCPS_ERR_INVALID_ARG, "bad n_frames");
    if (n_frames == 0) return SCPS_OK;
    if (!X || !V || !HV) return fail(SCPS_ERR_INVALID_ARG, "X, V and HV are required");
    const int nta = ((s->topos[topo].n + kTile - 1) / kTile) * kTile;
    SCPS_CU(launch_hvp(s->d.elec, s->d_topos + topo, s->base, X, V, HV, n_frames, nta,
                       (cudaStream_t)stream));
    return SCPS_OK;
}

int scps_collect_paths(scps_system* s, int32_t rep0, int32_t nrep, float* frames, double* z,
                       double* zmin, double* epot, double* bias_T, int64_t* n_frames_out) {
    TraceRange trace_("scps_collect_paths");
    if (!s) return fail(SCPS_ERR_INVALID_ARG, "NULL system");
    const int R = s->d.n_replicas;
    if (rep0 < 0 || nrep < 0 || rep0 + nrep > R) return fail(SCPS_ERR_INVALID_ARG, "replica range");
    SCPS_CU(cudaDeviceSynchronize());
    const int mf = std::max(s->d.max_frames, 1);
    const int dims = is_2d(s->model) ? 2 : 3;
    std::vector<long long> ns(R);
    SCPS_CU(cudaMemcpy(ns.data(), s->st.n_saved, sizeof(long long) * R, cudaMemcpyDeviceToHost));
    std::vector<double> buf((size_t)nrep * mf);
    double* dst[4] = {z, zmin, epot, bias_T};
    double* src[4] = {s->st.fz, s->st.fzm, s->st.fe, s->st.fT};
    for (int q = 0; q < 4; ++q) {
        if (!dst[q]) continue;
        SCPS_CU(cudaMemcpy(buf.data(), src[q] + (size_t)rep0 * mf, sizeof(double) * nrep * mf,
                           cudaMemcpyDeviceToHost));
        for (int k = 0; k < nrep; ++k) {
            const long long n_have = std::min<long long>(ns[rep0 + k], mf);
            const long long first = ns[rep0 + k] > mf ? ns[rep0 + k] % mf : 0;
            for (long long f = 0; f < n_have; ++f)
                dst[q][(size_t)k * mf + f] = buf[(size_t)k * mf + (first + f) % mf];
        }
    }
    if (frames && s->d.save_interval > 0) {
        size_t out_off = 0;
        for (int k = 0; k < nrep; ++k) {
            const int r = rep0 + k;
            const int n = atoms_per_replica(s, r);
            const size_t per = (size_t)n * dims;
            std::vector<float> fb((size_t)mf * per);
            const size_t src_off = is_2d(s->model) ? (size_t)r * mf * 2
                                                                : (size_t)s->frame_off[r] * 3;
            SCPS_CU(cudaMemcpy(fb.data(), s->st.frames + src_off, sizeof(float) * fb.size(),
                               cudaMemcpyDeviceToHost));
            const long long n_have = std::min<long long>(ns[r], mf);
            const long long first = ns[r] > mf ? ns[r] % mf : 0;
            for (long long f = 0; f < n_have; ++f)
                std::memcpy(frames + out_off + f * per, fb.data() + ((first + f) % mf) * per,
                            sizeof(float) * per);
            out_off += (size_t)mf * per;
        }
    }
    if (n_frames_out)
        for (int k = 0; k < nrep; ++k) n_frames_out[k] = std::min<long long>(ns[rep0 + k], mf);
    return SCPS_OK;
}

int scps_get_state(scps_system* s, double* x, double* v, double* zm, int64_t* step, double* bias_T) {
    TraceRange trace_("scps_get_state");
    if (!s) return fail(SCPS_ERR_INVALID_ARG, "NULL system");
    SCPS_CU(cudaDeviceSynchronize());
    const int R = s->d.n_replicas;
    if (is_2d(s->model)) {
        if (x) SCPS_CU(cudaMemcpy(x, s->st.xy, sizeof(double2) * R, cudaMemcpyDeviceToHost));
        if (v) std::memset(v, 0, sizeof(double) * 2 * R);
    } else if (s->is_box) {  // slots are in tile order: place each atom by its id
        const BoxDev& B = s->box;
        const size_t np = (size_t)R * B.np;
        std::vector<float4> hp(np), hv(np);
        std::vector<int> hid(np);
        SCPS_CU(cudaMemcpy(hid.data(), B.id, sizeof(int) * np, cudaMemcpyDeviceToHost));
        if (x) SCPS_CU(cudaMemcpy(hp.data(), B.pos, sizeof(float4) * np, cudaMemcpyDeviceToHost));
        if (v) SCPS_CU(cudaMemcpy(hv.data(), B.vel, sizeof(float4) * np, cudaMemcpyDeviceToHost));
        for (int r = 0; r < R; ++r)
            for (int q = 0; q < B.np; ++q) {
                const size_t sl = (size_t)r * B.np + q;
                const int a = hid[sl];
                if (a < 0) continue;
                const size_t o = 3 * ((size_t)r * B.n_atoms + a);
                if (x) {
                    x[o] = hp[sl].x;
                    x[o + 1] = hp[sl].y;
                    x[o + 2] = hp[sl].z;
                }
                if (v) {
                    v[o] = hv[sl].x;
                    v[o + 1] = hv[sl].y;
                    v[o + 2] = hv[sl].z;
                }
            }
    } else {
        std::vector<float4> h(s->n_atoms_total);
        if (x) {
            SCPS_CU(cudaMemcpy(h.data(), s->st.x, sizeof(float4) * h.size(), cudaMemcpyDeviceToHost));
            for (size_t i = 0; i < h.size(); ++i) {
                x[3 * i] = h[i].x;
                x[3 * i + 1] = h[i].y;
                x[3 * i + 2] = h[i].z;
            }
        }
        if (v) {
            SCPS_CU(cudaMemcpy(h.data(), s->st.v, sizeof(float4) * h.size(), cudaMemcpyDeviceToHost));
            for (size_t i = 0; i < h.size(); ++i) {
                v[3 * i] = h[i].x;
                v[3 * i + 1] = h[i].y;
                v[3 * i + 2] = h[i].z;
            }
        }
    }
    if (zm) SCPS_CU(cudaMemcpy(zm, s->st.zm, sizeof(double) * R, cudaMemcpyDeviceToHost));
    if (step) SCPS_CU(cudaMemcpy(step, s->st.step, sizeof(long long) * R, cudaMemcpyDeviceToHost));
    if (bias_T) SCPS_CU(cudaMemcpy(bias_T, s->st.T, sizeof(double) * R, cudaMemcpyDeviceToHost));
    return SCPS_OK;
}

int scps_set_state(scps_system* s, const double* x, const double* v, const double* zm,
                   const int64_t* step, const double* bias_T) {
    TraceRange trace_("scps_set_state");
    if (!s) return fail(SCPS_ERR_INVALID_ARG, "NULL system");
    SCPS_CU(cudaDeviceSynchronize());
    const int R = s->d.n_replicas;
    if (is_2d(s->model)) {
        if (x) {
            for (int r = 0; r < 2 * R; ++r)
                if (!std::isfinite(x[r])) return fail(SCPS_ERR_NONFINITE, "non-finite position");
            SCPS_CU(cudaMemcpy(s->st.xy, x, sizeof(double2) * R, cudaMemcpyHostToDevice));
        }
    } else if (s->is_box) {  // positions go in atom order; the next step rebuilds the lists
        const BoxDev& B = s->box;
        if (v && !x) return fail(SCPS_ERR_UNSUPPORTED, "the periodic box sets velocities with positions");
        if (x) {
            const size_t n3 = (size_t)3 * R * B.n_atoms;
            std::vector<float> hx(n3), hv(n3, 0.f);
            for (size_t i = 0; i < n3; ++i) {
                if (!std::isfinite(x[i]) || (v && !std::isfinite(v[i])))
                    return fail(SCPS_ERR_NONFINITE, "non-finite position or velocity");
                hx[i] = (float)x[i];
                if (v) hv[i] = (float)v[i];
            }
            float* dx = nullptr;
            SCPS_CU(cudaMalloc(&dx, sizeof(float) * n3));
            cudaError_t e = cudaMemcpy(dx, hx.data(), sizeof(float) * n3, cudaMemcpyHostToDevice);
            for (int r = 0; r < R && e == cudaSuccess; ++r)
                e = box_load(B, s->d_topos, s->st, dx + (size_t)3 * r * B.n_atoms, r, 0);
            if (e == cudaSuccess) e = cudaDeviceSynchronize();
            cudaFree(dx);
            SCPS_CU(e);
            // velocities: slots are in atom order right after the load
            std::vector<float4> h4((size_t)R * B.np, make_float4(0.f, 0.f, 0.f, 0.f));
            for (int r = 0; r < R; ++r)
                for (int a = 0; a < B.n_atoms; ++a) {
                    const size_t o = 3 * ((size_t)r * B.n_atoms + a);
                    h4[(size_t)r * B.np + a] = make_float4(hv[o], hv[o + 1], hv[o + 2], 0.f);
                }
            SCPS_CU(cudaMemcpy(B.vel, h4.data(), sizeof(float4) * h4.size(), cudaMemcpyHostToDevice));
        }
    } else {
        std::vector<float4> h(s->n_atoms_total);
        if (x) {
            for (size_t i = 0; i < h.size(); ++i) {
                for (int k = 0; k < 3; ++k)
                    if (!std::isfinite(x[3 * i + k]))
                        return fail(SCPS_ERR_NONFINITE, "non-finite position at packed atom %zu", i);
                h[i] = make_float4((float)x[3 * i], (float)x[3 * i + 1], (float)x[3 * i + 2], 0.f);
            }
            SCPS_CU(cudaMemcpy(s->st.x, h.data(), sizeof(float4) * h.size(), cudaMemcpyHostToDevice));
        }
        if (v) {
            for (size_t i = 0; i < h.size(); ++i) {
                for (int k = 0; k < 3; ++k)
                    if (!std::isfinite(v[3 * i + k]))
                        return fail(SCPS_ERR_NONFINITE, "non-finite velocity at packed atom %zu", i);
                h[i] = make_float4((float)v[3 * i], (float)v[3 * i + 1], (float)v[3 * i + 2], 0.f);
            }
            SCPS_CU(cudaMemcpy(s->st.v, h.data(), sizeof(float4) * h.size(), cudaMemcpyHostToDevice));
        }
    }
    if (zm) SCPS_CU(cudaMemcpy(s->st.zm, zm, sizeof(double) * R, cudaMemcpyHostToDevice));
    if (step) {
        for (int r = 0; r < R; ++r) {
            if (step[r] < 0 || step[r] > (int64_t)UINT32_MAX) return fail(SCPS_ERR_INVALID_ARG, "step out of range");
            s->host_step[r] = step[r];
        }
        SCPS_CU(cudaMemcpy(s->st.step, step, sizeof(long long) * R, cudaMemcpyHostToDevice));
    }
    if (bias_T) SCPS_CU(cudaMemcpy(s->st.T, bias_T, sizeof(double) * R, cudaMemcpyHostToDevice));
    if (x || v) {
        std::vector<int> zero(R, 0);
        SCPS_CU(cudaMemcpy(s->st.status, zero.data(), sizeof(int) * R, cudaMemcpyHostToDevice));
    }
    return SCPS_OK;
}

int scps_get_status(scps_system* s, int32_t* per_replica) {
    TraceRange trace_("scps_get_status");
    if (!s) return fail(SCPS_ERR_INVALID_ARG, "NULL system");
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return fail(SCPS_ERR_CUDA, "device error: %s", cudaGetErrorString(e));
    const int R = s->d.n_replicas;
    std::vector<int> st(R);
    SCPS_CU(cudaMemcpy(st.data(), s->st.status, sizeof(int) * R, cudaMemcpyDeviceToHost));
    int rc = SCPS_OK;
    for (int r = 0; r < R; ++r) {
        if (per_replica) per_replica[r] = st[r];
        if (st[r] & (SCPS_REPLICA_NONFINITE | SCPS_REPLICA_FORCE_RANGE)) rc = SCPS_ERR_NONFINITE;
        else if (st[r] != SCPS_REPLICA_OK && rc == SCPS_OK) rc = SCPS_ERR_LIST_OVERFLOW;
    }
    if (rc == SCPS_ERR_NONFINITE) fail(rc, "a replica produced non-finite or out-of-range values and was frozen");
    else if (rc) fail(rc, "a neighbour list overflowed and the replica was frozen");
    return rc;
}

int scps_get_info(const scps_system* s, scps_info* info) {
    if (!s || !info) return fail(SCPS_ERR_INVALID_ARG, "NULL argument");
    *info = s->info;
    info->n_replicas = s->d.n_replicas;
    info->n_atoms_total = s->n_atoms_total;
    info->max_atoms = s->max_atoms;
    info->cluster_size = s->cluster;
    info->threads = s->threads;
    info->steps_per_graph = s->steps_per_graph;
    info->launch_groups = (int32_t)s->groups.size();
    info->plan = s->plan;
    info->kernels_per_step_call = 1;
    info->device_bytes = s->bytes;
    info->pair_checks_per_step = 0;
    info->list_skin = s->list_skin;
    info->steps_per_list_build = 0.0;
    if (s->st.pair_slots && !s->is_box) {  // summed over replicas, from the lists each built last
        std::vector<long long> ps(s->d.n_replicas);
        std::vector<int> nb(s->d.n_replicas);
        SCPS_CU(cudaMemcpy(ps.data(), s->st.pair_slots, sizeof(long long) * ps.size(),
                           cudaMemcpyDeviceToHost));
        SCPS_CU(cudaMemcpy(nb.data(), s->st.list_builds, sizeof(int) * nb.size(),
                           cudaMemcpyDeviceToHost));
        double builds = 0.0;
        for (size_t r = 0; r < ps.size(); ++r) {
            info->pair_checks_per_step += ps[r];
            builds += nb[r];
        }
        if (builds > 0.0 && s->last_launch_steps > 0)
            info->steps_per_list_build = (double)s->last_launch_steps * (double)ps.size() / builds;
    }
    if (s->is_box) {  // 64 pair slots per chunk of 8 entries, from the lists built last
        SCPS_CU(cudaDeviceSynchronize());
        const size_t ncl = (size_t)s->d.n_replicas * 4 * s->box.nt;
        std::vector<int> ne(ncl);
        SCPS_CU(cudaMemcpy(ne.data(), s->box.nent, sizeof(int) * ncl, cudaMemcpyDeviceToHost));
        long long slots = 0;
        for (int v : ne) slots += 8ll * v;
        info->pair_checks_per_step = slots;
        // list builds and rebuild steps of the latest step call
        const int R = s->d.n_replicas;
        std::vector<int> nb(R);
        int nev = 0;
        SCPS_CU(cudaMemcpy(nb.data(), s->box.nbuild, sizeof(int) * (size_t)R, cudaMemcpyDeviceToHost));
        SCPS_CU(cudaMemcpy(&nev, s->box.nevent, sizeof(int), cudaMemcpyDeviceToHost));
        double builds = 0.0;
        for (int v : nb) builds += v;
        if (builds > 0.0 && s->last_launch_steps > 0)
            info->steps_per_list_build = (double)s->last_launch_steps * (double)R / builds;
        info->graph_nodes_last_call += 8ll * nev;
    }
    return SCPS_OK;
}

int scps_path_average(scps_system* s, int32_t n_sel, const int32_t* replicas, int32_t n_frames,
                      double* out) {
    TraceRange trace_("scps_path_average");
    if (!s || !replicas || !out) return fail(SCPS_ERR_INVALID_ARG, "NULL argument");
    if (!is_2d(s->model) && (s->model != SCPS_MODEL_CHAIN || s->is_box))
        return fail(SCPS_ERR_UNSUPPORTED, "path averages cover the two-dimensional models and chains");
    const int R = s->d.n_replicas, mf = s->d.max_frames;
    if (n_sel < 1 || n_frames < 1 || n_frames > mf)
        return fail(SCPS_ERR_INVALID_ARG, "need n_sel >= 1 and 1 <= n_frames <= max_frames");
    std::vector<long long> ns(R);
    SCPS_CU(cudaMemcpy(ns.data(), s->st.n_saved, sizeof(long long) * R, cudaMemcpyDeviceToHost));
    std::vector<int> sel(replicas, replicas + n_sel);
    for (int r : sel) {
        if (r < 0 || r >= R) return fail(SCPS_ERR_INVALID_ARG, "replica %d out of range", r);
        if (ns[r] < n_frames || ns[r] > mf)
            return fail(SCPS_ERR_STATE, "replica %d holds %lld frames (needs %d, at most %d kept)", r,
                        ns[r], n_frames, mf);
    }
    if (s->model == SCPS_MODEL_CHAIN) {  // average contact maps
        const int t = s->rep_topo[sel[0]];
        for (int r : sel)
            if (s->rep_topo[r] != t) return fail(SCPS_ERR_INVALID_ARG, "selected replicas differ in topology");
        const int nc = s->topos[t].ncon, n = s->topos[t].n;
        if (nc < 1 || !s->topos[t].dev.con_ij)
            return fail(SCPS_ERR_STATE, "contact maps need the contact list of a contact or tube bias");
        std::vector<long long> fo(n_sel);
        for (int q = 0; q < n_sel; ++q) fo[q] = s->frame_off[sel[q]];
        long long* d_fo = nullptr;
        double* d_out = nullptr;
        const size_t nout = (size_t)n_frames * nc;
        cudaError_t e = cudaMalloc(&d_fo, sizeof(long long) * n_sel);
        if (e == cudaSuccess) e = cudaMalloc(&d_out, sizeof(double) * nout);
        if (e == cudaSuccess) e = cudaMemcpy(d_fo, fo.data(), sizeof(long long) * n_sel, cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = launch_path_average_contacts(s->st, s->topos[t].dev.con_ij, nc, n, d_fo, n_sel, n_frames,
                                             (double)s->inv_r0sq, d_out, 0);
        if (e == cudaSuccess) e = cudaMemcpy(out, d_out, sizeof(double) * nout, cudaMemcpyDeviceToHost);
        cudaFree(d_fo);
        cudaFree(d_out);
        if (e != cudaSuccess) return fail(SCPS_ERR_CUDA, "path average failed: %s", cudaGetErrorString(e));
        return SCPS_OK;
    }
    int* d_sel = nullptr;
    double2* d_out = nullptr;
    cudaError_t e = cudaMalloc(&d_sel, sizeof(int) * n_sel);
    if (e == cudaSuccess) e = cudaMalloc(&d_out, sizeof(double2) * n_frames);
    if (e == cudaSuccess) e = cudaMemcpy(d_sel, sel.data(), sizeof(int) * n_sel, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_path_average_2d(s->st, mf, n_frames, d_sel, n_sel, d_out, 0);
    if (e == cudaSuccess) e = cudaMemcpy(out, d_out, sizeof(double2) * n_frames, cudaMemcpyDeviceToHost);
    cudaFree(d_sel);
    cudaFree(d_out);
    if (e != cudaSuccess) return fail(SCPS_ERR_CUDA, "path average failed: %s", cudaGetErrorString(e));
    return SCPS_OK;
}

// Autotuner of the periodic box: pair-list skin x rebuild cadence, each probed for
// probe_steps steps on the system itself from a device snapshot of the box state (slot
// order, positions, velocities, ids and the per-replica scalars); every probe and the final
// restore force a list rebuild, since a list built for a smaller skin does not cover the
// displacements a larger one allows.
static int box_autotune(scps_system* s, int probe_steps, int use_cache, scps_tune_result* out) {
    BoxDev& B = s->box;
    const int R = s->d.n_replicas;
    int n_sm = 0;
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, s->device);
    const std::string key = "box|" + std::to_string(n_sm) + "|" + std::to_string(s->d.elec) + "|" +
                            std::to_string(B.n_atoms) + "x" + std::to_string(R);
    static std::mutex mu;
    static std::map<std::string, std::pair<double, int>> cache;  // skin, rebuild_every
    const double rc = s->base.pc.rc > 0.f ? (double)s->base.pc.rc : 1.0;
    std::vector<int> ones(R, 1);
    auto apply = [&](double skin, int every) {
        s->box_graphs.reset();  // the step graphs hold the box parameters by value
        s->list_skin = skin;
        B.rebuild_every = every;
        B.rlist2 = (float)((rc + skin) * (rc + skin));
        B.skin2_quarter = (float)(0.25 * skin * skin);
        return cudaMemcpyAsync(B.need, ones.data(), sizeof(int) * R, cudaMemcpyHostToDevice,
                               s->cap_stream);
    };
    scps_tune_result res{};
    res.plan = s->plan;
    res.cluster_size = 1;
    res.threads = 0;
    res.skin = s->list_skin;
    res.rebuild_every = B.rebuild_every;
    if (use_cache) {
        bool hit = false;
        std::pair<double, int> c;
        {
            std::lock_guard<std::mutex> lk(mu);
            auto it = cache.find(key);
            if (it != cache.end()) {
                hit = true;
                c = it->second;
            }
        }
        if (hit) {
            SCPS_CU(apply(c.first, c.second));
            SCPS_CU(cudaStreamSynchronize(s->cap_stream));
            res.skin = c.first;
            res.rebuild_every = c.second;
            res.from_cache = 1;
            if (out) *out = res;
            return SCPS_OK;
        }
    }
    // device snapshot of what a probe changes
    const size_t np = (size_t)R * B.np;
    struct Region {
        void* p;
        size_t n;
    };
    const Region regions[] = {
        {B.pos, sizeof(float4) * np},          {B.vel, sizeof(float4) * np},
        {B.id, sizeof(int) * np},              {B.par, sizeof(float2) * np},
        {B.slot_of, sizeof(int) * (size_t)R * B.n_atoms},
        {B.pos_ref, sizeof(float4) * np},      {B.since, sizeof(int) * R},
        {B.maxd2, sizeof(unsigned) * R},       {B.eb, sizeof(double) * R},
        {s->st.zm, sizeof(double) * R},        {s->st.z, sizeof(double) * R},
        {s->st.T, sizeof(double) * R},         {s->st.step, sizeof(long long) * R},
        {s->st.status, sizeof(int) * R}};
    size_t total = 0;
    for (const Region& g : regions) total += (g.n + 255) & ~(size_t)255;
    unsigned char* snap = nullptr;
    SCPS_CU(cudaMalloc(&snap, total));
    auto copy_all = [&](bool save) -> cudaError_t {
        size_t off = 0;
        cudaError_t c = cudaSuccess;
        for (const Region& g : regions) {
            if (c == cudaSuccess)
                c = cudaMemcpyAsync(save ? (void*)(snap + off) : g.p, save ? g.p : (void*)(snap + off),
                                    g.n, cudaMemcpyDeviceToDevice, s->cap_stream);
            off += (g.n + 255) & ~(size_t)255;
        }
        if (c == cudaSuccess) c = cudaStreamSynchronize(s->cap_stream);
        return c;
    };
    cudaError_t e = copy_all(true);
    if (e != cudaSuccess) {
        cudaFree(snap);
        return fail(SCPS_ERR_CUDA, "tuner snapshot failed: %s", cudaGetErrorString(e));
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    RunParams P = s->base;
    P.save_interval = 0;
    const long long frame_atoms = (long long)std::max(s->d.max_frames, 1) * B.n_atoms;
    const long long step0 = s->host_step[0];
    // returns us per step, or -2e300 when a restore failed
    auto probe = [&](double skin, int every) -> double {
        cudaError_t le = apply(skin, every);
        if (le == cudaSuccess)
            le = box_run(B, s->d_topos, s->st, P, s->d_rep_ids, R, s->d.elec, s->ncon_max, step0,
                         std::max(1, probe_steps / 4), frame_atoms, &s->box_graphs, s->cap_stream);
        if (le == cudaSuccess) le = copy_all(false);
        if (le == cudaSuccess) le = apply(skin, every);
        if (le == cudaSuccess) le = cudaEventRecord(e0, s->cap_stream);
        if (le == cudaSuccess)
            le = box_run(B, s->d_topos, s->st, P, s->d_rep_ids, R, s->d.elec, s->ncon_max, step0,
                         probe_steps, frame_atoms, &s->box_graphs, s->cap_stream);
        if (le == cudaSuccess) le = cudaEventRecord(e1, s->cap_stream);
        if (le == cudaSuccess) le = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (le == cudaSuccess) le = cudaEventElapsedTime(&ms, e0, e1);
        std::vector<int> stat(R, 0);  // a frozen replica (e.g. a list overflow) voids the probe
        if (le == cudaSuccess)
            le = cudaMemcpy(stat.data(), s->st.status, sizeof(int) * R, cudaMemcpyDeviceToHost);
        if (copy_all(false) != cudaSuccess || le != cudaSuccess) return -2e300;
        for (int r = 0; r < R; ++r)
            if (stat[r] != 0) return -1.0;
        return 1e3 * ms / probe_steps;
    };
    const double skin0 = s->list_skin;
    const int every0 = B.rebuild_every;
    std::vector<std::pair<double, int>> cands{{skin0, every0}};
    for (double sk : {0.1, 0.15, 0.2})
        for (int ev : {10, 20, 40})
            if (std::fabs(sk - skin0) > 1e-9 || ev != every0) cands.push_back({sk, ev});
    double best = 1e300;
    std::pair<double, int> best_c = cands[0];
    int timed = 0;
    for (size_t k = 0; k < cands.size(); ++k) {
        const double us = probe(cands[k].first, cands[k].second);
        if (us < -1e300) {
            apply(skin0, every0);
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            cudaFree(snap);
            return fail(SCPS_ERR_CUDA, "tuner probe or restore failed");
        }
        if (us < 0.0) continue;
        ++timed;
        if (k == 0) res.us_per_step_initial = us;
        if (us < 0.98 * best) {  // more than 2 % faster, as for the chains
            best = us;
            best_c = cands[k];
        }
    }
    e = apply(best_c.first, best_c.second);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->cap_stream);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(snap);
    SCPS_CU(e);
    {
        std::lock_guard<std::mutex> lk(mu);
        cache[key] = best_c;
    }
    res.skin = best_c.first;
    res.rebuild_every = best_c.second;
    res.candidates = timed;
    res.us_per_step = best;
    if (out) *out = res;
    return SCPS_OK;
}

int scps_autotune(scps_system* s, int32_t probe_steps, int32_t use_cache, scps_tune_result* out) {
    TraceRange trace_("scps_autotune");
    if (!s) return fail(SCPS_ERR_INVALID_ARG, "NULL system");
    if (probe_steps < 1 || probe_steps > 100000) return fail(SCPS_ERR_INVALID_ARG, "probe_steps outside [1, 1e5]");
    if (s->model == SCPS_MODEL_CHAIN && s->is_box) {
        for (int r = 1; r < s->d.n_replicas; ++r)
            if (s->host_step[r] != s->host_step[0])
                return fail(SCPS_ERR_STATE, "periodic-box replicas must share one step counter");
        return box_autotune(s, probe_steps, use_cache, out);
    }
    if (s->model != SCPS_MODEL_CHAIN || s->d.exec != SCPS_EXEC_RESIDENT)
        return fail(SCPS_ERR_UNSUPPORTED, "the tuner covers the resident form of chain replicas and the periodic box");
    const int R = s->d.n_replicas;
    int n_sm = 0;
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, s->device);
    // cache key: SM count, electrostatics, bias kind and the multiset of replica sizes
    std::map<int, int> sizes;
    for (int r = 0; r < R; ++r) sizes[s->topos[s->rep_topo[r]].n] += 1;
    std::string key = std::to_string(n_sm) + "|" + std::to_string(s->d.elec) + "|" +
                      std::to_string(s->bias_kind);
    for (auto& kv : sizes) key += "|" + std::to_string(kv.first) + "x" + std::to_string(kv.second);
    static std::mutex mu;
    static std::map<std::string, std::vector<int>> cache;  // plan, cluster, threads, skin (pm)
    scps_tune_result res{};
    res.plan = s->plan;
    res.cluster_size = s->cluster;
    res.threads = s->threads;
    res.skin = s->list_skin;
    res.rebuild_every = s->base.rebuild_every;
    if (use_cache) {
        std::vector<int> hit;
        {
            std::lock_guard<std::mutex> lk(mu);
            auto it = cache.find(key);
            if (it != cache.end()) hit = it->second;
        }
        if (!hit.empty()) {
            int rc = set_groups(s, hit[0], hit[1], hit[2]);
            if (rc) return rc;
            set_skin(s, 1e-3 * hit[3]);
            drop_graphs(s);
            res.plan = hit[0];
            res.cluster_size = hit[1];
            res.threads = hit[2];
            res.skin = s->list_skin;
            res.from_cache = 1;
            if (out) *out = res;
            return SCPS_OK;
        }
    }
    // snapshot of the state the probes change (no frames are saved while probing)
    const size_t na = (size_t)s->n_atoms_total;
    float4 *sx = nullptr, *sv = nullptr;
    double *szm = nullptr, *sz = nullptr, *sT = nullptr;
    long long* sstep = nullptr;
    int* sstat = nullptr;
    auto release = [&]() {
        cudaFree(sx); cudaFree(sv); cudaFree(szm); cudaFree(sz); cudaFree(sT); cudaFree(sstep);
        cudaFree(sstat);
    };
    cudaError_t e = cudaMalloc(&sx, sizeof(float4) * na);
    if (e == cudaSuccess) e = cudaMalloc(&sv, sizeof(float4) * na);
    if (e == cudaSuccess) e = cudaMalloc(&szm, sizeof(double) * R);
    if (e == cudaSuccess) e = cudaMalloc(&sz, sizeof(double) * R);
    if (e == cudaSuccess) e = cudaMalloc(&sT, sizeof(double) * R);
    if (e == cudaSuccess) e = cudaMalloc(&sstep, sizeof(long long) * R);
    if (e == cudaSuccess) e = cudaMalloc(&sstat, sizeof(int) * R);
    auto copy_all = [&](bool save) -> cudaError_t {
        cudaError_t c = cudaSuccess;
        auto cp = [&](void* a, void* b, size_t n) {
            if (c == cudaSuccess) c = cudaMemcpyAsync(save ? a : b, save ? b : a, n, cudaMemcpyDeviceToDevice, s->cap_stream);
        };
        cp(sx, s->st.x, sizeof(float4) * na);
        cp(sv, s->st.v, sizeof(float4) * na);
        cp(szm, s->st.zm, sizeof(double) * R);
        cp(sz, s->st.z, sizeof(double) * R);
        cp(sT, s->st.T, sizeof(double) * R);
        cp(sstep, s->st.step, sizeof(long long) * R);
        cp(sstat, s->st.status, sizeof(int) * R);
        if (c == cudaSuccess) c = cudaStreamSynchronize(s->cap_stream);
        return c;
    };
    if (e == cudaSuccess) e = copy_all(true);
    if (e != cudaSuccess) {
        release();
        return fail(SCPS_ERR_CUDA, "tuner snapshot failed: %s", cudaGetErrorString(e));
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    RunParams P = s->base;
    P.save_interval = 0;
    const int initial[3] = {s->plan, s->cluster, s->threads};
    std::vector<std::vector<int>> cands;
    cands.push_back({initial[0], initial[1], initial[2]});
    const int n_plans = sizes.size() > 1 ? 2 : 1;
    for (int plan = 0; plan < n_plans; ++plan)
        for (int cl : {1, 2})
            for (int th : {256, 512, cl == 2 ? kMaxThreadsPair : 1024}) {
                std::vector<int> c{plan, cl, th};
                if (c != cands[0]) cands.push_back(c);
            }
    const size_t smem_limit = resident_smem_limit();
    double best = 1e300;
    std::vector<int> best_c = cands[0];
    int timed = 0;
    // one short untimed run (first-launch set-up), then the timed probe; the state is
    // restored after each. Returns the time per step in us, or a negative value when the
    // launch was refused (the candidate is skipped); a failed restore is fatal (-2e300).
    auto probe = [&](const RunParams& Pp) -> double {
        cudaError_t le = launch_groups(s, Pp, std::max(1, probe_steps / 4), s->cap_stream);
        if (le == cudaSuccess) le = copy_all(false);
        if (le == cudaSuccess) le = cudaEventRecord(e0, s->cap_stream);
        if (le == cudaSuccess) le = launch_groups(s, Pp, probe_steps, s->cap_stream);
        if (le == cudaSuccess) le = cudaEventRecord(e1, s->cap_stream);
        if (le == cudaSuccess) le = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (le == cudaSuccess) le = cudaEventElapsedTime(&ms, e0, e1);
        if (copy_all(false) != cudaSuccess) return -2e300;
        if (le != cudaSuccess) {
            (void)cudaGetLastError();  // a launch-configuration error
            return -1.0;
        }
        return 1e3 * ms / probe_steps;
    };
    auto abort_restore = [&]() {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        release();
        return fail(SCPS_ERR_CUDA, "tuner restore failed");
    };
    for (size_t k = 0; k < cands.size(); ++k) {
        const std::vector<int>& c = cands[k];
        if (set_groups(s, c[0], c[1], c[2]) != SCPS_OK) continue;
        bool fits = true;
        for (auto& g : s->groups)
            fits = fits && resident_smem_bytes(g.nta) <= smem_limit;
        if (!fits) continue;
        const double us = probe(P);
        if (us < -1e300) return abort_restore();
        if (us < 0.0) continue;
        ++timed;
        if (k == 0) res.us_per_step_initial = us;
        // a candidate must win by more than 2 %: a shape within the timing noise of a
        // short probe does not replace the current one (or an earlier candidate)
        if (us < 0.98 * best) {
            best = us;
            best_c = c;
        }
    }
    int rc = set_groups(s, best_c[0], best_c[1], best_c[2]);
    if (rc) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        release();
        return rc;
    }
    // list skin at the chosen shape: a larger skin adds pairs to every step and makes
    // list builds rarer (the cadence follows from the displacement bound). Forces do not
    // depend on it, so every choice gives the same trajectory bit for bit.
    double best_skin = s->list_skin;
    for (double sk : {0.06, 0.09, 0.12, 0.16, 0.2}) {
        if (std::fabs(sk - s->list_skin) < 1e-9) continue;
        const double keep = s->list_skin;
        set_skin(s, sk);
        RunParams Ps = s->base;
        Ps.save_interval = 0;
        const double us = probe(Ps);
        set_skin(s, keep);
        if (us < -1e300) return abort_restore();
        if (us < 0.0) continue;
        ++timed;
        if (us < 0.98 * best) {
            best = us;
            best_skin = sk;
        }
    }
    set_skin(s, best_skin);
    drop_graphs(s);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    release();
    best_c.push_back((int)std::lround(1e3 * best_skin));
    {
        std::lock_guard<std::mutex> lk(mu);
        cache[key] = best_c;
    }
    res.plan = best_c[0];
    res.cluster_size = best_c[1];
    res.threads = best_c[2];
    res.skin = best_skin;
    res.candidates = timed;
    res.us_per_step = best;
    if (out) *out = res;
    return SCPS_OK;
}

int scps_philox4x32_10(int64_t n, const uint32_t* ctr, uint32_t key0, uint32_t key1, uint32_t* out,
                       void* stream) {
    if (n < 0 || (n > 0 && (!ctr || !out))) return fail(SCPS_ERR_INVALID_ARG, "bad arguments");
    SCPS_CU(launch_philox(n, ctr, key0, key1, out, (cudaStream_t)stream));
    return SCPS_OK;
}

}  // extern "C"

// Accessors for the allocation-free entry point (noalloc.cu).
namespace scps {
int internal_topology(const scps_system* s, int topo, TopoDev* out, int* elec, RunParams* P) {
    if (s->model != SCPS_MODEL_CHAIN) return fail(SCPS_ERR_UNSUPPORTED, "chain model only");
    if (s->is_box)  // its kernels take every pair once, with no periodic images
        return fail(SCPS_ERR_UNSUPPORTED,
                    "the allocation-free evaluation covers open-boundary chains, not periodic boxes");
    if (topo < 0 || topo >= (int)s->topos.size())
        return fail(SCPS_ERR_INVALID_ARG, "bad topology %d", topo);
    *out = s->topos[topo].dev;
    *elec = s->d.elec;
    *P = s->base;
    return SCPS_OK;
}

int internal_fail(int code, const char* msg) { return fail(code, "%s", msg); }
}  // namespace scps
