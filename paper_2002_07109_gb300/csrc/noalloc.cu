// Pair energies without any device allocation.
//
// Some callers cannot call cudaMalloc: code that lives inside an allocator
// owning the whole device pool (a caching allocator would see a foreign
// allocation it cannot account for), hosts that forbid allocation after
// start-up (embedded or real-time loops, where cudaMalloc may block and
// synchronise the device), and plug-ins that are handed device buffers but
// no allocation rights.  For them, bounce_pair_energy_noalloc computes the
// same Coulomb and Lennard-Jones pair energy totals as the energy kernel of a
// context (bounce_get_energies), but over all pairs of a caller-supplied
// state and with its scratch in a file-scope device array instead of context
// buffers.
//
// Scratch: g_noalloc_scratch below, BOUNCE_NOALLOC_MAX_ATOMS atoms
// (48 bytes per atom: split FP32 positions and two per-atom FP64 partial
// sums, 786,432 bytes in all), plus one status word, held by every GPU that
// loads this library until the process exits.  Host code cannot use the
// array's name as a device address (on the host it names a shadow
// variable), so the first call on each device looks the address up with
// cudaGetSymbolAddress while that device is current and keeps it; make that
// first call before any stream capture.  Every call overwrites every
// per-atom slot it reads and clears the status word first, so nothing else
// needs clearing between calls; calls whose GPU work overlaps (two streams,
// two threads) share the array and race.
#include <cmath>
#include <mutex>

#include <math_constants.h>

#include "../../include/bounce.h"
#include "common.cuh"

namespace {

constexpr int NOALLOC_MAX = BOUNCE_NOALLOC_MAX_ATOMS;
// per atom: two float4 and two doubles; then one status word (bad type seen)
constexpr size_t NOALLOC_BYTES = (size_t)NOALLOC_MAX * (2 * sizeof(float4) + 2 * sizeof(double)) + 256;
constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

std::mutex g_mu;
void* g_scratch_ptr[MAX_DEVICES] = {nullptr};

struct Layout {
    float4* hi;
    float4* lo;
    double* part;  // [2][n]: coulomb, lj per atom
    int* bad;      // set when an atom type lies outside [0, n_types)
};

__host__ __device__ inline Layout layout(void* base, int n) {
    Layout l;
    l.hi = (float4*)base;
    l.lo = l.hi + NOALLOC_MAX;
    l.part = (double*)(l.lo + NOALLOC_MAX);
    l.bad = (int*)(l.part + 2 * (size_t)NOALLOC_MAX);
    (void)n;
    return l;
}

// Clears the status word (one thread); the pack kernel that follows on the
// same stream may then flag bad types.
__global__ void k_na_clear(void* scratch) { *layout(scratch, 0).bad = 0; }

// Split FP32 copies of the positions.  A type outside [0, n_types) would
// index the LJ tables out of bounds: it is replaced by type 0 here and
// flagged, and k_na_sum then writes NaN to both totals.
__global__ void k_na_pack(void* scratch, int n, const double* q, const double* charge, const int* type, int n_types,
                          Params p) {
    Layout l = layout(scratch, n);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double x = q[3 * (size_t)i], y = q[3 * (size_t)i + 1], z = q[3 * (size_t)i + 2];
        if (p.periodic) {
            x -= p.Ld[0] * floor(x / p.Ld[0]);
            y -= p.Ld[1] * floor(y / p.Ld[1]);
            z -= p.Ld[2] * floor(z / p.Ld[2]);
        }
        const float hx = __double2float_rn(x), hy = __double2float_rn(y), hz = __double2float_rn(z);
        int t = type[i];
        if (t < 0 || t >= n_types) {
            atomicOr(l.bad, 1);
            t = 0;
        }
        l.hi[i] = make_float4(hx, hy, hz, (float)charge[i]);
        l.lo[i] = make_float4(__double2float_rn(x - (double)hx), __double2float_rn(y - (double)hy),
                              __double2float_rn(z - (double)hz), __int_as_float(t));
    }
}

// Exact FP64 r^2 from the caller's (n, 3) positions (same operations as the
// context path).
__device__ __forceinline__ double na_exact_r2(const Params& p, const double* q, int i, int j) {
    double d[3];
    for (int c = 0; c < 3; ++c) {
        d[c] = __dsub_rn(q[3 * (size_t)i + c], q[3 * (size_t)j + c]);
        if (p.periodic) d[c] = __dsub_rn(d[c], __dmul_rn(p.Ld[c], rint(__ddiv_rn(d[c], p.Ld[c]))));
    }
    return __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
}

// One warp per atom i sums W over j > i of another molecule inside r_c.
__global__ void k_na_pairs(void* scratch, int n, const double* q, const int* mol, Params p) {
    Layout l = layout(scratch, n);
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= n) return;
    const float4 hi = l.hi[i], lo = l.lo[i];
    const int ti = type_of(lo), mi = mol[i];
    float ec = 0.f, el = 0.f;
    for (int j = i + 1 + lane; j < n; j += 32) {
        if (mol[j] == mi) continue;
        const float4 hj = l.hi[j], lj = l.lo[j];
        const float3 d = pair_disp(p, hi, lo, hj, lj);
        const float r2 = d.x * d.x + d.y * d.y + d.z * d.z;
        bool in = r2 < p.rc2_lo;
        if (!in && r2 <= p.rc2_hi) in = na_exact_r2(p, q, i, j) < p.rc2_d;
        if (in) {
            float a, b;
            pair_W(p, r2, p.kcoul * hi.w * hj.w, ti * BOUNCE_MAXT + type_of(lj), a, b);
            ec += a;
            el += b;
        }
    }
    double dc = ec, dl = el;
    for (int o = 16; o > 0; o >>= 1) {
        dc += __shfl_xor_sync(0xffffffffu, dc, o);
        dl += __shfl_xor_sync(0xffffffffu, dl, o);
    }
    if (lane == 0) {
        l.part[i] = dc;
        l.part[NOALLOC_MAX + i] = dl;
    }
}

// Fixed-order sum of the per-atom partial sums into out[2] (one CTA).
__global__ void k_na_sum(void* scratch, int n, double kfix, double* out) {
    Layout l = layout(scratch, n);
    __shared__ double part[2][256];
    for (int t = 0; t < 2; ++t) {
        double acc = 0.0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) acc += l.part[(size_t)t * NOALLOC_MAX + i];
        part[t][threadIdx.x] = acc;
    }
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            part[0][threadIdx.x] += part[0][threadIdx.x + w];
            part[1][threadIdx.x] += part[1][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const bool bad = *l.bad != 0;
        out[0] = bad ? CUDART_NAN : kfix * part[0][0];
        out[1] = bad ? CUDART_NAN : part[1][0];
    }
}

}  // namespace

extern "C" int bounce_pair_energy_noalloc(int32_t n, const double* q, const double* charge, const int32_t* type,
                                          const int32_t* molecule, int32_t n_types, const double* sigma,
                                          const double* eps, double r_cut, double ewald_beta, const double* box,
                                          double* out, void* stream) {
    if (n < 1 || n > NOALLOC_MAX || !q || !charge || !type || !molecule || !out || n_types < 1 ||
        n_types > BOUNCE_MAXT || !sigma || !eps || ewald_beta < 0)
        return BOUNCE_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return BOUNCE_ERR_CUDA;
    void* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_scratch_ptr[dev]) {
            void* ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return BOUNCE_ERR_CUDA;
            g_scratch_ptr[dev] = ptr;
        }
        scratch = g_scratch_ptr[dev];
    }
    // the same scalar parameters as a context's energy kernel (no device memory)
    Params p{};
    for (int a = 0; a < n_types; ++a)
        for (int b = 0; b < n_types; ++b) {
            const double s6 = std::pow(sigma[a * n_types + b], 6);
            p.c12[a * BOUNCE_MAXT + b] = (float)(4.0 * eps[a * n_types + b] * s6 * s6);
            p.c6[a * BOUNCE_MAXT + b] = (float)(4.0 * eps[a * n_types + b] * s6);
        }
    p.kcoul = (float)KCOUL_D;
    const bool cut = std::isfinite(r_cut) && r_cut > 0;
    const double rc2 = cut ? r_cut * r_cut : INFINITY;
    p.rc2_lo = cut ? (float)(rc2 * (1.0 - 1e-5)) : INFINITY;
    p.rc2_hi = cut ? (float)(rc2 * (1.0 + 1e-5)) : INFINITY;
    p.rc2_d = rc2;
    p.ebeta = (float)ewald_beta;
    p.e2b_sqrtpi = (float)(2.0 * ewald_beta / std::sqrt(M_PI));
    p.periodic = box ? 1 : 0;
    for (int d = 0; d < 3; ++d) {
        const double Lb = box ? box[d] : 1.0;
        if (!(Lb > 0)) return BOUNCE_ERR_INVALID_ARG;
        // minimum image: beyond half an edge the sum would no longer be the pair sum
        if (box && !(cut && 2.0 * r_cut <= Lb)) return BOUNCE_ERR_INVALID_ARG;
        p.Ld[d] = Lb;
        p.iLd[d] = 1.0 / Lb;
        p.Lhi[d] = (float)Lb;
        p.Llo[d] = (float)(Lb - (double)p.Lhi[d]);
        p.invL[d] = (float)(1.0 / Lb);
    }
    cudaStream_t st = (cudaStream_t)stream;
    // an error left pending by earlier, unrelated work is not this call's:
    // refuse to launch rather than report (and clear) it as our own
    if (cudaPeekAtLastError() != cudaSuccess) return BOUNCE_ERR_CUDA;
    k_na_clear<<<1, 1, 0, st>>>(scratch);
    if (cudaGetLastError() != cudaSuccess) return BOUNCE_ERR_CUDA;
    k_na_pack<<<(n + 255) / 256, 256, 0, st>>>(scratch, n, q, charge, type, n_types, p);
    if (cudaGetLastError() != cudaSuccess) return BOUNCE_ERR_CUDA;
    k_na_pairs<<<(n + 7) / 8, 256, 0, st>>>(scratch, n, q, molecule, p);
    if (cudaGetLastError() != cudaSuccess) return BOUNCE_ERR_CUDA;
    k_na_sum<<<1, 256, 0, st>>>(scratch, n, KCOUL_D / (double)p.kcoul, out);
    return cudaGetLastError() == cudaSuccess ? BOUNCE_OK : BOUNCE_ERR_CUDA;
}
