// Pair sums over all pairs (droplets and batches of replicas without a
// cutoff; the F_0 share of every pair, Sec. IV.A / V, and BAOAB's full pair
// gradient).
//
// Work: a static list of items (replica, i-tile of 32 atoms, j-block of tj
// atoms of the same replica at or after the i-tile), built on the host when
// the topology or the replica layout is set; every unordered pair of a
// replica lies in exactly one item (two atoms of one tile: in the item whose
// j-block starts at that tile, with j > i).  A resident grid of warps
// strides over the items: lane l holds atom i0 + l, the j-block is staged in
// shared memory 32 atoms at a time, and in sub-step k lane l evaluates its
// pair with atom (l + k) mod 32 of the stage.  Both sides of every pair are
// summed once (Newton's third law): the i side in the lane's registers, the j
// side in a register that moves to the next lane after every sub-step, so
// that after 32 sub-steps lane l holds the sum of atom l of the stage; both
// go to int64 fixed-point accumulators (2^-32 kcal/mol/A) rounded from FP32
// by the int64 conversion, so the result does not depend on the order in
// which warps finish.  The j-block length tj is chosen by the autotuner
// (bounce_autotune).
#include "common.cuh"

namespace {

__device__ __forceinline__ void tl_add(unsigned long long* a, float v) {
    if (v != 0.f) atomicAdd(a, fix_round<32>(v));
}

template <int PART>
__global__ void __launch_bounds__(256) k_tile_pairs(DevSys s, Params p, int step_off) {
    chain_enter();
    __shared__ float4 sh_h[8][32], sh_l[8][32];
    __shared__ int sh_m[8][32];
    __shared__ float s_c12[BOUNCE_MAXT * BOUNCE_MAXT], s_c6[BOUNCE_MAXT * BOUNCE_MAXT];
    if (threadIdx.x < BOUNCE_MAXT * BOUNCE_MAXT) {  // LJ table: per-lane type pairs read from shared memory
        s_c12[threadIdx.x] = p.c12[threadIdx.x];
        s_c6[threadIdx.x] = p.c6[threadIdx.x];
    }
    __syncthreads();
    const DevTile& t = s.tl;
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const int cur = (int)((*s.step_base + step_off) & 1);
    const size_t n = (size_t)s.n;
    int npair = 0;
    for (int it = blockIdx.x * 8 + wl; it < t.nitems; it += gridDim.x * 8) {
        const int4 w = t.items[it];  // (first i, number of i, first j, number of j)
        const bool vi = lane < w.y;
        const int i = w.x + lane;
        float4 hi = make_float4(0.f, 0.f, 0.f, 0.f), lo = hi;
        int mi = -1;
        if (vi) {
            hi = s.phi[cur][i];
            lo = s.plo[cur][i];
            mi = s.mol[i];
        }
        const float qi = p.kcoul * hi.w;
        const int ti = type_of(lo) * BOUNCE_MAXT;
        float gix = 0.f, giy = 0.f, giz = 0.f;
        for (int jb = 0; jb < w.w; jb += 32) {
            const int nj = min(32, w.w - jb), j0 = w.z + jb;
            __syncwarp();
            if (lane < nj) {
                sh_h[wl][lane] = s.phi[cur][j0 + lane];
                sh_l[wl][lane] = s.plo[cur][j0 + lane];
                sh_m[wl][lane] = s.mol[j0 + lane];
            } else {  // padding: finite zeros, masked below
                sh_h[wl][lane] = make_float4(0.f, 0.f, 0.f, 0.f);
                sh_l[wl][lane] = make_float4(0.f, 0.f, 0.f, 0.f);
                sh_m[wl][lane] = -1;
            }
            __syncwarp();
            float ax = 0.f, ay = 0.f, az = 0.f;  // j-side sum of stage atom (lane + k) mod 32
#pragma unroll 4
            for (int k = 0; k < 32; ++k) {
                const int m = (lane + k) & 31;
                const float4 hj = sh_h[wl][m], lj = sh_l[wl][m];
                const int mj = sh_m[wl][m];
                const float3 d = pair_disp(p, hi, lo, hj, lj);
                const float r2 = d.x * d.x + d.y * d.y + d.z * d.z;
                const bool in = mj >= 0 && mi >= 0 && mi != mj && j0 + m > i;
                const int tp = ti + type_of(lj);
                const float w0 = pairsum_w<PART>(p, in ? r2 : 1.f, qi * hj.w, s_c12[tp], s_c6[tp]);
                const float wv = in ? w0 : 0.f;
                npair += in ? 1 : 0;
                gix = fmaf(wv, d.x, gix);
                giy = fmaf(wv, d.y, giy);
                giz = fmaf(wv, d.z, giz);
                ax = fmaf(-wv, d.x, ax);
                ay = fmaf(-wv, d.y, ay);
                az = fmaf(-wv, d.z, az);
                // the j-side sum moves to the lane that meets its atom next
                const int from = (lane + 1) & 31;
                ax = __shfl_sync(0xffffffffu, ax, from);
                ay = __shfl_sync(0xffffffffu, ay, from);
                az = __shfl_sync(0xffffffffu, az, from);
            }
            if (lane < nj) {
                const size_t jj = (size_t)(j0 + lane);
                tl_add(t.acc + jj, ax);
                tl_add(t.acc + n + jj, ay);
                tl_add(t.acc + 2 * n + jj, az);
            }
        }
        if (vi) {
            tl_add(t.acc + i, gix);
            tl_add(t.acc + n + i, giy);
            tl_add(t.acc + 2 * n + i, giz);
        }
    }
    npair = warp_sum_i(npair);
    if (lane == 0 && npair) atomicAdd(&s.cnt[PART == 3 ? CNT_SHORT_PAIRS : CNT_FULL_PAIRS], (unsigned long long)npair);
}

// Accumulated sums added to out (n x 3, FP64); accumulators cleared.
__global__ void k_tile_collect(DevSys s, double* out) {
    const size_t n = (size_t)s.n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < s.n; i += gridDim.x * blockDim.x)
        for (int d = 0; d < 3; ++d) {
            const long long v = (long long)s.tl.acc[d * n + i];
            s.tl.acc[d * n + i] = 0ull;
            out[3 * (size_t)i + d] += (double)v * CL_UNFIX;
        }
}

}  // namespace

void launch_tile_pairs(const DevSys& s, const Params& p, int step_off, int part, cudaStream_t st) {
    const int blocks = std::max(1, std::min(s.tl.blocks, (s.tl.nitems + 7) / 8));
    if (part == 3) launch_chained(k_tile_pairs<3>, blocks, 256, 0, st, s, p, step_off);
    else launch_chained(k_tile_pairs<5>, blocks, 256, 0, st, s, p, step_off);
}

void launch_tile_collect(const DevSys& s, double* out, cudaStream_t st) {
    k_tile_collect<<<(s.n + 255) / 256, 256, 0, st>>>(s, out);
}
