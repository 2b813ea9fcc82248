// Observables of the paper's accuracy study (Sec. VI): pair-distance
// histograms for radial distribution functions and mean-square
// displacement for the Einstein self-diffusion coefficient.
//
// Histogram: one warp per atom i of type ta or tb walks its candidate row
// (members j > i of the matching type), takes the bin from the FP32 distance
// and re-decides in FP64 against the squared FP64 bin edges (k w)^2 when the
// distance lies within 1e-5 relative of an edge, so bin counts match an
// FP64 evaluation exactly.  Counts are 64-bit integer atomics (order-free).
#include "common.cuh"

namespace {

__device__ __forceinline__ double edge_sq(double w, int k) {
    const double e = __dmul_rn((double)k, w);
    return __dmul_rn(e, e);
}

__global__ void k_pair_hist(DevSys s, Params p, int cur, int ta, int tb, float inv_w, double w, int n_bins,
                            unsigned long long* hist) {
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= s.n) return;
    const float4 hi = s.phi[cur][i], lo = s.plo[cur][i];
    const int ti = type_of(lo);
    if (ti != ta && ti != tb) return;
    const int n = s.nlong[i];
    const int* row = s.rows + (size_t)i * s.cap;
    const double rmax2 = edge_sq(w, n_bins);
    for (int k = lane; k < n; k += 32) {
        const int j = row[k];
        if (j <= i) continue;
        const float4 hj = s.phi[cur][j], lj = s.plo[cur][j];
        const int tj = type_of(lj);
        if (!((ti == ta && tj == tb) || (ti == tb && tj == ta))) continue;
        const float3 d = pair_disp(p, hi, lo, hj, lj);
        const float r = sqrtf(d.x * d.x + d.y * d.y + d.z * d.z);
        const float x = r * inv_w;
        int b = (int)x;
        const float fr = x - (float)b;
        if (fr < 1e-4f || fr > 1.f - 1e-4f || b >= n_bins - 1) {
            const double r2 = exact_r2(s, p, cur, i, j);
            if (!(r2 < rmax2)) continue;
            b = max(0, min(b, n_bins - 1));
            while (b > 0 && r2 < edge_sq(w, b)) --b;
            while (b < n_bins - 1 && r2 >= edge_sq(w, b + 1)) ++b;
        }
        if (b < n_bins) atomicAdd(&hist[b], 1ull);
    }
}

__global__ void k_msd_terms(DevSys s, const double* rx, const double* ry, const double* rz, int cur, int t,
                            double* terms) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < s.n; i += gridDim.x * blockDim.x) {
        double v = 0.0, c = 0.0;
        if (s.type[i] == t) {
            const double dx = s.qx[cur][i] - rx[i], dy = s.qy[cur][i] - ry[i], dz = s.qz[cur][i] - rz[i];
            v = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
            c = 1.0;
        }
        terms[i] = v;
        terms[s.n + i] = c;
    }
}

__global__ void k_sum2(int n, const double* terms, double* out) {
    __shared__ double part[2][256];
    for (int t = 0; t < 2; ++t) {
        double acc = 0.0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) acc += terms[(size_t)t * n + i];
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
    if (threadIdx.x < 2) out[threadIdx.x] = part[threadIdx.x][0];
}

}  // namespace

void launch_pair_hist(const DevSys& s, const Params& p, int cur, int ta, int tb, double r_max, int n_bins,
                      unsigned long long* hist, cudaStream_t st) {
    const double w = r_max / n_bins;
    const int wpb = 8;
    k_pair_hist<<<(s.n + wpb - 1) / wpb, wpb * 32, 0, st>>>(s, p, cur, ta, tb, (float)(1.0 / w), w, n_bins, hist);
}

void launch_msd(const DevSys& s, const double* rx, const double* ry, const double* rz, int cur, int t,
                double* terms, cudaStream_t st) {
    k_msd_terms<<<(s.n + 255) / 256, 256, 0, st>>>(s, rx, ry, rz, cur, t, terms);
    k_sum2<<<1, 256, 0, st>>>(s.n, terms, terms + 2 * (size_t)s.n);
}
