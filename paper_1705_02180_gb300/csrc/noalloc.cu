// Allocation-free energy/force evaluation of one configuration.
//
// Some callers cannot call cudaMalloc at the moment they need forces: code
// that runs while a CUDA stream is being captured into a graph (allocation is
// not allowed inside a global-mode capture), frameworks that have reserved the
// whole device memory for their own pool, and latency-critical loops where a
// device allocation (and the implicit synchronisation it may cause) is not
// acceptable. scps_energy_forces_noalloc serves them: it evaluates U and F of
// one configuration with the plain-form pair and bonded kernels, accumulating
// into a fixed scratch array that lives in this file for the lifetime of the
// process instead of in memory allocated per call.
//
// Forces and the energy are summed in 64-bit fixed point (units of 2^-20) with
// integer atomics, so the result does not depend on the order in which threads
// add their terms: repeated calls on the same X give the same bits. Each thread
// sums its own atom's pair terms in FP32 in a fixed j order before converting.
// Only open-boundary chains are evaluated (periodic boxes are refused).
//
// The scratch is a file-scope __device__ array (every GPU that loads the
// library holds it until the process exits). Host code must not pass the
// array's name to a kernel: on the host that name is only a stand-in, so its
// device address is looked up with cudaGetSymbolAddress once per device.
#include <mutex>

#include "../../include/scps.h"
#include "scps_internal.h"

namespace scps {
int internal_topology(const scps_system* s, int topo, TopoDev* out, int* elec, RunParams* P);
int internal_fail(int code, const char* msg);
}  // namespace scps

namespace scps {
namespace {

constexpr int kNoAllocMaxAtoms = 8192;  // largest topology the static scratch holds
constexpr int kMaxDevices = 64;

// Force components (SoA, 3 x kNoAllocMaxAtoms) and the energy, fixed point 2^-20.
struct NoAllocScratch {
    unsigned long long F[3 * kNoAllocMaxAtoms];
    unsigned long long E[32];
};

__device__ __forceinline__ void na_add(unsigned long long* a, float v) {
    atomicAdd(a, (unsigned long long)f2fix(v));
}
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

std::mutex g_setup_mutex;
NoAllocScratch* g_scratch_ptr[kMaxDevices] = {};

__global__ void k_na_clear(NoAllocScratch* sc, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 3 * n) sc->F[i] = 0ull;
    if (i == 0) sc->E[0] = 0ull;
}

template <int ELEC>
__global__ void k_na_pairs(const float* __restrict__ X, NoAllocScratch* sc, TopoDev tp,
                           RunParams P) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = tp.n_atoms;
    if (i >= n) return;
    unsigned long long* F = sc->F;
    const float xi = X[3 * i], yi = X[3 * i + 1], zi = X[3 * i + 2];
    const float qi = tp.qs[i];
    const float2 li = tp.lj[i];
    const unsigned long long em = tp.excl[i];
    float fx = 0.f, fy = 0.f, fz = 0.f, e = 0.f;
    for (int j = i + 1; j < n; ++j) {
        const int dj = j - i + kExclWindow;
        if (dj < 2 * kExclWindow && ((em >> dj) & 1ull)) continue;
        const float dx = X[3 * j] - xi, dy = X[3 * j + 1] - yi, dz = X[3 * j + 2] - zi;
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        if (r2 >= P.pc.rc2) continue;
        const float2 lj = tp.lj[j];
        float ep = 0.f;
        const float s = pair_s<ELEC, true>(r2, li.x + lj.x, li.y * lj.y, qi * tp.qs[j], P.pc, &ep);
        fx = fmaf(s, dx, fx);
        fy = fmaf(s, dy, fy);
        fz = fmaf(s, dz, fz);
        na_add(&F[j], -s * dx);
        na_add(&F[n + j], -s * dy);
        na_add(&F[2 * n + j], -s * dz);
        e += ep;
    }
    na_add(&F[i], fx);
    na_add(&F[n + i], fy);
    na_add(&F[2 * n + i], fz);
    na_add(&sc->E[0], e);
}

__global__ void k_na_bonded(const float* __restrict__ X, NoAllocScratch* sc, TopoDev tp) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = tp.n_atoms;
    unsigned long long* F = sc->F;
    if (t < tp.n_bonds) {
        const int2 ij = tp.bond_ij[t];
        const float2 par = tp.bond_par[t];
        const float dx = X[3 * ij.y] - X[3 * ij.x], dy = X[3 * ij.y + 1] - X[3 * ij.x + 1],
                    dz = X[3 * ij.y + 2] - X[3 * ij.x + 2];
        const float r = sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
        const float dr = r - par.x;
        const float f = par.y * dr / r;
        na_add(&F[ij.x], f * dx);
        na_add(&F[n + ij.x], f * dy);
        na_add(&F[2 * n + ij.x], f * dz);
        na_add(&F[ij.y], -f * dx);
        na_add(&F[n + ij.y], -f * dy);
        na_add(&F[2 * n + ij.y], -f * dz);
        na_add(&sc->E[0], 0.5f * par.y * dr * dr);
    } else if (t < tp.n_bonds + tp.n_angles) {
        const int q = t - tp.n_bonds;
        const int4 ijk = tp.ang_ijk[q];
        const float2 par = tp.ang_par[q];
        const float ux = X[3 * ijk.x] - X[3 * ijk.y], uy = X[3 * ijk.x + 1] - X[3 * ijk.y + 1],
                    uz = X[3 * ijk.x + 2] - X[3 * ijk.y + 2];
        const float wx = X[3 * ijk.z] - X[3 * ijk.y], wy = X[3 * ijk.z + 1] - X[3 * ijk.y + 1],
                    wz = X[3 * ijk.z + 2] - X[3 * ijk.y + 2];
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
        na_add(&F[ijk.x], fix);
        na_add(&F[n + ijk.x], fiy);
        na_add(&F[2 * n + ijk.x], fiz);
        na_add(&F[ijk.z], fkx);
        na_add(&F[n + ijk.z], fky);
        na_add(&F[2 * n + ijk.z], fkz);
        na_add(&F[ijk.y], -(fix + fkx));
        na_add(&F[n + ijk.y], -(fiy + fky));
        na_add(&F[2 * n + ijk.y], -(fiz + fkz));
        na_add(&sc->E[0], 0.5f * par.y * dth * dth);
    }
}

// Scratch (SoA) -> caller's F (n x 3) and U.
__global__ void k_na_finish(const NoAllocScratch* sc, int n, float* __restrict__ F,
                            double* __restrict__ U) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && F) {
        F[3 * i] = fix2f((long long)sc->F[i]);
        F[3 * i + 1] = fix2f((long long)sc->F[n + i]);
        F[3 * i + 2] = fix2f((long long)sc->F[2 * n + i]);
    }
    if (i == 0) *U = (double)(long long)sc->E[0] * 9.5367431640625e-07;  // 2^-20
}

// Device address of the scratch for the current device (looked up once per device).
int scratch_for_current_device(NoAllocScratch** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return internal_fail(SCPS_ERR_CUDA, "no usable current CUDA device");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return internal_fail(SCPS_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed");
        g_scratch_ptr[dev] = (NoAllocScratch*)p;
    }
    *out = g_scratch_ptr[dev];
    return SCPS_OK;
}

}  // namespace
}  // namespace scps

using namespace scps;

extern "C" int scps_energy_forces_noalloc(scps_system* s, int32_t topo, const float* X,
                                          double* U, float* F, void* stream) {
    if (!s || !X || !U) return internal_fail(SCPS_ERR_INVALID_ARG, "NULL system, X or U");
    TopoDev tp;
    int elec = 0;
    RunParams P;
    int rc = internal_topology(s, topo, &tp, &elec, &P);
    if (rc) return rc;
    if (tp.n_atoms > kNoAllocMaxAtoms)
        return internal_fail(SCPS_ERR_UNSUPPORTED,
                             "scps_energy_forces_noalloc holds at most 8192 atoms per topology");
    NoAllocScratch* sc = nullptr;
    rc = scratch_for_current_device(&sc);
    if (rc) return rc;
    cudaStream_t cs = (cudaStream_t)stream;
    const int n = tp.n_atoms, th = 128;
    k_na_clear<<<(3 * n + th - 1) / th, th, 0, cs>>>(sc, n);
    const int gb = (n + th - 1) / th;
    switch (elec) {
        case ELEC_DDIEL: k_na_pairs<ELEC_DDIEL><<<gb, th, 0, cs>>>(X, sc, tp, P); break;
        case ELEC_RF: k_na_pairs<ELEC_RF><<<gb, th, 0, cs>>>(X, sc, tp, P); break;
        case ELEC_PLAIN: k_na_pairs<ELEC_PLAIN><<<gb, th, 0, cs>>>(X, sc, tp, P); break;
        default: k_na_pairs<ELEC_NONE><<<gb, th, 0, cs>>>(X, sc, tp, P); break;
    }
    const int nbt = tp.n_bonds + tp.n_angles;
    if (nbt > 0) k_na_bonded<<<(nbt + th - 1) / th, th, 0, cs>>>(X, sc, tp);
    k_na_finish<<<gb, th, 0, cs>>>(sc, n, F, U);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return internal_fail(SCPS_ERR_CUDA, cudaGetErrorString(e));
    return SCPS_OK;
}
