// Pair sums over clusters of atoms (the F_0 share of every pair, Sec. IV.A /
// Sec. V, and BAOAB's full pair gradient), for systems with a finite cutoff.
//
// Build (four gated launches; each returns at once unless the cluster
// rebuild flag is raised -- the step kernel raises it when an atom has moved
// more than skin/2 since the build):
//   1. column of every atom on a grid over (x, y), counts; the CTA finishing
//      last scans the counts;
//   2. scatter of the atom indices into column order;
//   3. one CTA per column sorts its atoms by (z, index) (bitonic sort in
//      shared memory: the order, hence every cluster, is deterministic),
//      cuts them into clusters of BOUNCE_CL and writes the slot-ordered
//      copies of the split positions, the molecule ids, the slot of every
//      atom and the bounding box of every cluster;
//   4. one warp per cluster I collects the atoms of the clusters J >= I of
//      the columns in reach that lie within the search radius of I's box
//      (minimum image per axis), in a fixed order, with the periodic image
//      of each; the CTA finishing last clears the flag and raises the prune
//      flag.
// Prune (a fifth gated launch, also raised by the step kernel when an atom
// has moved half the prune skin since the last prune): the entries of each
// list within r + prune skin of some atom of I at the current positions,
// so that the pair kernel reads a list close to the pairs it must evaluate
// while the outer lists, with a larger skin, are rebuilt rarely.
// Pair kernel: one warp per work item (cluster I, chunk of BOUNCE_CL_EPW
// pruned entries); lane = one list atom j, the 8 atoms
// of cluster I in turn from shared memory.  Every unordered pair inside the
// cutoff is evaluated once (Newton's third law): the j-side sum of a lane is
// added once per item, the i-side sums are reduced over the warp at the end
// of the item, both into int64 fixed-point accumulators (2^-32 kcal/mol/A)
// rounded from FP32 by the int64 conversion: integer addition is
// associative, so the result does not depend on the order in which warps
// finish.
#include <algorithm>
#include <cstdint>

#include "common.cuh"

namespace {

// resident CTAs per SM the pair kernel is compiled for (register budget)
#ifndef CL_PAIRS_MIN_CTAS
#define CL_PAIRS_MIN_CTAS 3
#endif

constexpr int CL = BOUNCE_CL;
constexpr int EPW = BOUNCE_CL_EPW;
constexpr int SORT_NT = 256;
constexpr int NO_SHIFT = 13;  // image code (kx + 1) * 9 + (ky + 1) * 3 + (kz + 1) of k = 0
constexpr int PER_PAIR = 31;  // the pair's clusters may straddle half a box edge: minimum image per atom pair

__device__ __forceinline__ bool cl_pending(const DevSys& s, int force) {
    chain_enter();
    return force || *s.cl.rebuild;
}

// True in the one CTA of the grid that finishes last; it resets the counter.
__device__ bool cl_last_cta(unsigned int* ctr) {
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        last = atomicAdd(ctr, 1u) == gridDim.x - 1;
        if (last) atomicExch(ctr, 0u);
    }
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// Exclusive block-wide scan of x over all threads of the CTA (blockDim a
// multiple of 32, at most 1024); returns the prefix, *total the sum.
__device__ int block_scan(int x, int* total) {
    __shared__ int wsum[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int v = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    if (lane == 31) wsum[w] = v;
    __syncthreads();
    if (w == 0) {
        int t = lane < nw ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        wsum[lane] = t;
    }
    __syncthreads();
    const int excl = (w > 0 ? wsum[w - 1] : 0) + v - x;
    *total = wsum[nw - 1];
    __syncthreads();
    return excl;
}

__device__ __forceinline__ int column_of(const DevClu& c, const Params& p, float4 hi) {
    int cx, cy;
    if (p.periodic) {
        cx = min(max((int)(hi.x * c.ihx), 0), c.ncx - 1);
        cy = min(max((int)(hi.y * c.ihy), 0), c.ncy - 1);
    } else {
        cx = min(max((int)floorf((hi.x - c.ox) * c.ihx), 0), c.ncx - 1);
        cy = min(max((int)floorf((hi.y - c.oy) * c.ihy), 0), c.ncy - 1);
    }
    return cy * c.ncx + cx;
}

// 1. columns and their counts; the last CTA scans them.
__global__ void k_cl_count(DevSys s, Params p, int step_off, int force) {
    if (!cl_pending(s, force)) return;
    const DevClu& c = s.cl;
    const int cur = (int)((*s.step_base + step_off) & 1);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < s.n; i += gridDim.x * blockDim.x) {
        const int col = column_of(c, p, s.phi[cur][i]);
        c.atom_col[i] = col;
        atomicAdd(&c.col_count[col], 1);
    }
    if (!cl_last_cta(&c.done_ctr[0])) return;
    int carry = 0;
    for (int b = 0; b < c.ncol; b += blockDim.x) {
        const int col = b + threadIdx.x;
        const int v = col < c.ncol ? __ldcg(&c.col_count[col]) : 0;
        int tot;
        const int ex = block_scan(v, &tot);
        if (col < c.ncol) {
            c.col_start[col] = carry + ex;
            c.col_fill[col] = carry + ex;
            c.col_count[col] = 0;
        }
        carry += tot;
    }
    if (threadIdx.x == 0) c.col_start[c.ncol] = carry;
}

// 2. atom indices in column order (arbitrary order inside a column).
__global__ void k_cl_scatter(DevSys s, Params p, int step_off, int force) {
    if (!cl_pending(s, force)) return;
    const DevClu& c = s.cl;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < s.n; i += gridDim.x * blockDim.x) {
        const int pos = atomicAdd(&c.col_fill[c.atom_col[i]], 1);
        c.col_atoms[pos] = i;
    }
}

// Order-preserving map of a float onto an unsigned key.
__device__ __forceinline__ uint32_t float_key(float z) {
    const uint32_t b = __float_as_uint(z);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// 3. one CTA per column: sort by (z, index), clusters, slots, boxes.
__global__ void __launch_bounds__(SORT_NT) k_cl_sort(DevSys s, Params p, int step_off, int force) {
    if (!cl_pending(s, force)) return;
    __shared__ unsigned long long key[BOUNCE_CL_MAXCOL];
    const DevClu& c = s.cl;
    const int tid = threadIdx.x;
    const int cur = (int)((*s.step_base + step_off) & 1);
    for (int col = blockIdx.x; col < c.ncol; col += gridDim.x) {
        const int b = c.col_start[col];
        int nc = c.col_start[col + 1] - b;
        if (nc > c.maxcol) {  // the column outgrew its capacity: the state is reported invalid
            if (tid == 0) atomicOr(s.err, BERR_LIST_OVERFLOW);
            nc = c.maxcol;
        }
        int P = 1;
        while (P < nc) P <<= 1;
        for (int t = tid; t < P; t += SORT_NT) {
            unsigned long long k = ~0ull;
            if (t < nc) {
                const int a = c.col_atoms[b + t];
                k = ((unsigned long long)float_key(s.phi[cur][a].z) << 32) | (uint32_t)a;
            }
            key[t] = k;
        }
        __syncthreads();
        for (int k = 2; k <= P; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int t = tid; t < P; t += SORT_NT) {
                    const int l = t ^ j;
                    if (l > t) {
                        const unsigned long long x = key[t], y = key[l];
                        if ((x > y) == ((t & k) == 0)) {
                            key[t] = y;
                            key[l] = x;
                        }
                    }
                }
                __syncthreads();
            }
        const int ncl = (nc + CL - 1) / CL;
        if (tid == 0) c.col_ncl[col] = ncl;
        for (int t = tid; t < ncl * CL; t += SORT_NT) {
            const int slot = (col * c.maxcl + t / CL) * CL + t % CL;
            if (t < nc) {
                const int a = (int)(uint32_t)(key[t] & 0xFFFFFFFFull);
                c.cl_atom[slot] = a;
                c.a2s[a] = slot;
                c.sphi[cur][slot] = s.phi[cur][a];
                c.splo[cur][slot] = s.plo[cur][a];
                c.smol[slot] = s.mol[a];
                const double qa = s.qx[cur][a], qb = s.qy[cur][a], qc = s.qz[cur][a];
                c.crefx[a] = qa;
                c.crefy[a] = qb;
                c.crefz[a] = qc;
                // the image of the wrapped copy in phi (the step kernel's wrap)
                c.cofx[a] = p.periodic ? p.Ld[0] * floor(qa / p.Ld[0]) : 0.0;
                c.cofy[a] = p.periodic ? p.Ld[1] * floor(qb / p.Ld[1]) : 0.0;
                c.cofz[a] = p.periodic ? p.Ld[2] * floor(qc / p.Ld[2]) : 0.0;
            } else {
                c.cl_atom[slot] = -1;
                c.smol[slot] = -1;
                c.sphi[cur][slot] = make_float4(0.f, 0.f, 0.f, 0.f);
                c.splo[cur][slot] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        for (int k = tid; k < ncl; k += SORT_NT) {
            float4 lo = make_float4(INFINITY, INFINITY, INFINITY, 0.f), hi = make_float4(-INFINITY, -INFINITY, -INFINITY, 0.f);
            for (int u = k * CL; u < min(nc, (k + 1) * CL); ++u) {
                const float4 h = s.phi[cur][(int)(uint32_t)(key[u] & 0xFFFFFFFFull)];
                lo.x = fminf(lo.x, h.x);
                lo.y = fminf(lo.y, h.y);
                lo.z = fminf(lo.z, h.z);
                hi.x = fmaxf(hi.x, h.x);
                hi.y = fmaxf(hi.y, h.y);
                hi.z = fmaxf(hi.z, h.z);
            }
            c.bb_lo[col * c.maxcl + k] = lo;
            c.bb_hi[col * c.maxcl + k] = hi;
        }
        __syncthreads();
    }
}

// Range of columns along one axis that a box [a, b] (extended by the search
// radius) meets: [lo, hi] on the unwrapped grid; `all` when it covers every
// column (periodic wrap would visit one twice).
__device__ __forceinline__ void column_span(int n, float a, float b, float org, float ih, int periodic, int& lo,
                                            int& hi, bool& all) {
    const float fa = (a - org) * ih, fb = (b - org) * ih;
    if (periodic) {
        lo = (int)floorf(fa);
        hi = (int)floorf(fb);
        all = hi - lo + 1 >= n;
        if (all) {
            lo = 0;
            hi = n - 1;
        }
    } else {
        lo = min(max((int)floorf(fa), 0), n - 1);
        hi = min(max((int)floorf(fb), 0), n - 1);
        all = false;
    }
}

// q_j - k L in split form (sh, sl: the high and low parts of k L): the high
// part rounded, its rounding error moved into the low part (two-sum), so the
// pair stays an exact split of the shifted coordinate.
__device__ __forceinline__ void shift_split(float& h, float& l, float sh, float sl) {
    const float t = h - sh;
    const float bb = t - h;
    const float err = (h - (t - bb)) + (-sh - bb);
    h = t;
    l = (l - sl) + err;
}

// 4. neighbour lists (warp per cluster I): every atom j of a cluster
// J >= I of the columns in reach whose distance to I's bounding box (minimum
// image per axis) is below the search radius, in a fixed order, as its slot
// with the periodic image of the pair (or the per-pair code when the pair's
// separation could reach half a box edge).  Every unordered pair of atoms
// inside the cutoff then appears once: in the list of the lower cluster, and
// for two atoms of one cluster with the lower slot as i.
__global__ void __launch_bounds__(256) k_cl_search(DevSys s, Params p, int step_off, int force) {
    if (!cl_pending(s, force)) return;
    const DevClu& c = s.cl;
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    const int ncl = c.ncol * c.maxcl;
    const int cur = (int)((*s.step_base + step_off) & 1);
    const float Lx = p.Lhi[0], Ly = p.Lhi[1], Lz = p.Lhi[2];
    bool overflow = false;
    for (int I = blockIdx.x * wpb + (threadIdx.x >> 5); I < ncl; I += gridDim.x * wpb) {
        const int col = I / c.maxcl, k = I - col * c.maxcl;
        if (k >= c.col_ncl[col]) {
            if (lane == 0) {
                c.lcnt[0][I] = 0;
                c.lcnt[1][I] = 0;
            }
            continue;
        }
        const float4 lo = c.bb_lo[I], hi = c.bb_hi[I];
        const float cx = 0.5f * (lo.x + hi.x), cy = 0.5f * (lo.y + hi.y), cz = 0.5f * (lo.z + hi.z);
        const float ex = 0.5f * (hi.x - lo.x), ey = 0.5f * (hi.y - lo.y), ez = 0.5f * (hi.z - lo.z);
        const float R = c.rsx[0];
        int xa, xb, ya, yb;
        bool xall, yall;
        column_span(c.ncx, lo.x - R, hi.x + R, p.periodic ? 0.f : c.ox, c.ihx, p.periodic, xa, xb, xall);
        column_span(c.ncy, lo.y - R, hi.y + R, p.periodic ? 0.f : c.oy, c.ihy, p.periodic, ya, yb, yall);
        int m0 = 0, m1 = 0;
        const uint32_t below = (1u << lane) - 1u;
        for (int yy = ya; yy <= yb; ++yy) {
            const int cyn = p.periodic ? (yy % c.ncy + c.ncy) % c.ncy : yy;
            for (int xx = xa; xx <= xb; ++xx) {
                const int cxn = p.periodic ? (xx % c.ncx + c.ncx) % c.ncx : xx;
                const int coln = cyn * c.ncx + cxn;
                const int colb = coln * c.maxcl;
                // the clusters J >= I of the column: all of them, or those after I in I's own column
                const int nk = c.col_ncl[coln];
                const int k0 = colb > I ? 0 : (colb == I - k ? k : nk);
                for (int kb = k0; kb < nk; kb += 32) {
                    // cluster level: boxes within the search radius (minimum image per axis)
                    const int kk = kb + lane;
                    bool near = false;
                    if (kk < nk) {
                        const float4 lj = c.bb_lo[colb + kk], hj = c.bb_hi[colb + kk];
                        float dx = cx - 0.5f * (lj.x + hj.x), dy = cy - 0.5f * (lj.y + hj.y),
                              dz = cz - 0.5f * (lj.z + hj.z);
                        if (p.periodic) {
                            dx -= rintf(dx * p.invL[0]) * Lx;
                            dy -= rintf(dy * p.invL[1]) * Ly;
                            dz -= rintf(dz * p.invL[2]) * Lz;
                        }
                        const float gx = fmaxf(fabsf(dx) - (ex + 0.5f * (hj.x - lj.x)), 0.f);
                        const float gy = fmaxf(fabsf(dy) - (ey + 0.5f * (hj.y - lj.y)), 0.f);
                        const float gz = fmaxf(fabsf(dz) - (ez + 0.5f * (hj.z - lj.z)), 0.f);
                        near = gx * gx + gy * gy + gz * gz < c.rs2[0];
                    }
                    uint32_t qual = __ballot_sync(0xffffffffu, near);
                    // atom level, four qualifying clusters per pass: lane = 8 q + t
                    while (qual) {
                        int pick = -1;
                        uint32_t rest = qual;
                        for (int q = 0; q <= (lane >> 3); ++q) {
                            pick = rest ? __ffs(rest) - 1 : -1;
                            rest = rest ? rest & (rest - 1) : 0u;
                        }
                        for (int q = 0; q < 4 && qual; ++q) qual &= qual - 1;
                        const int sj = pick >= 0 ? (colb + kb + pick) * CL + (lane & 7) : 0;
                        bool inL = false, inS = false;
                        int code = NO_SHIFT;
                        if (pick >= 0 && c.smol[sj] >= 0) {
                            const float4 h = c.sphi[cur][sj];
                            float dx = h.x - cx, dy = h.y - cy, dz = h.z - cz;
                            if (p.periodic) {
                                const int kx = (int)rintf(dx * p.invL[0]);
                                const int ky = (int)rintf(dy * p.invL[1]);
                                const int kz = (int)rintf(dz * p.invL[2]);
                                dx -= kx * Lx;
                                dy -= ky * Ly;
                                dz -= kz * Lz;
                                // image code of q_j - k L (the kernel subtracts k L from q_j)
                                code = (kx + 1) * 9 + (ky + 1) * 3 + (kz + 1);
                                if (fabsf(dx) + 2.f * ex >= 0.49f * Lx || fabsf(dy) + 2.f * ey >= 0.49f * Ly ||
                                    fabsf(dz) + 2.f * ez >= 0.49f * Lz)
                                    code = PER_PAIR;
                            }
                            const float gx = fmaxf(fabsf(dx) - ex, 0.f), gy = fmaxf(fabsf(dy) - ey, 0.f),
                                        gz = fmaxf(fabsf(dz) - ez, 0.f);
                            const float d2 = gx * gx + gy * gy + gz * gz;
                            inL = d2 < c.rs2[0];
                            inS = c.nlists > 1 && d2 < c.rs2[1];
                        }
                        const uint32_t bl = __ballot_sync(0xffffffffu, inL), bs = __ballot_sync(0xffffffffu, inS);
                        const int ent = sj | (code << 27);
                        if (inL) {
                            const int pos = m0 + __popc(bl & below);
                            if (pos < c.capj[0]) c.lst[0][(size_t)I * c.capj[0] + pos] = ent;
                        }
                        if (inS) {
                            const int pos = m1 + __popc(bs & below);
                            if (pos < c.capj[1]) c.lst[1][(size_t)I * c.capj[1] + pos] = ent;
                        }
                        m0 += __popc(bl);
                        m1 += __popc(bs);
                    }
                }
            }
        }
        if (lane == 0) {
            c.lcnt[0][I] = min(m0, c.capj[0]);
            c.lcnt[1][I] = c.nlists > 1 ? min(m1, c.capj[1]) : 0;
        }
        overflow = overflow || m0 > c.capj[0] || (c.nlists > 1 && m1 > c.capj[1]);
    }
    if (overflow) atomicOr(s.err, BERR_LIST_OVERFLOW);
    if (!cl_last_cta(&c.done_ctr[1])) return;
    if (threadIdx.x == 0) {
        *c.rebuild = 0;
        *c.prune = 1;  // new lists: prune them before the next pair sums
    }
}

// Whether list entry `ent` (high part hj of the j atom's slot copy) lies
// within sqrt(R2) of some atom of the cluster in shi/slo: high parts with the
// entry's periodic image (their rounding is far below the radius's margin),
// or the per-pair minimum image from the split positions (rare).
__device__ __forceinline__ bool prune_keep(const DevSys& s, const Params& p, int cur, int ent, float4 hj,
                                           const float4* shi, const float4* slo, float R2) {
    const DevClu& c = s.cl;
    const int sj = ent & 0x07FFFFFF, code = (int)((uint32_t)ent >> 27);
    float best = INFINITY;
    if (code == PER_PAIR) {
        const float4 lj = c.splo[cur][sj];
        for (int a = 0; a < CL; ++a) {
            const float3 d = pair_disp(p, shi[a], slo[a], hj, lj);
            best = fminf(best, d.x * d.x + d.y * d.y + d.z * d.z);
        }
    } else {
        if (code != NO_SHIFT) {
            hj.x -= (float)(code / 9 - 1) * p.Lhi[0];
            hj.y -= (float)((code / 3) % 3 - 1) * p.Lhi[1];
            hj.z -= (float)(code % 3 - 1) * p.Lhi[2];
        }
#pragma unroll
        for (int a = 0; a < CL; ++a) {
            const float dx = shi[a].x - hj.x, dy = shi[a].y - hj.y, dz = shi[a].z - hj.z;
            best = fminf(best, dx * dx + dy * dy + dz * dz);
        }
    }
    return best < R2;
}

// 5. pruned lists (warp per cluster I), gated by the prune flag: the
// entries of each list whose atom j lies within the prune radius of at least
// one atom of I at the current positions (same images as the pair kernel;
// FP32 with a margin, so that no pair the exact test would keep is dropped),
// in list order.  The step kernel raises the flag when an atom's slot copy has moved half the
// prune skin since this launch, which it records here.
__global__ void __launch_bounds__(256) k_cl_prune(DevSys s, Params p, int step_off, int force) {
    chain_enter();
    if (!(force || *s.cl.prune)) return;
    const DevClu& c = s.cl;
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5, wl = threadIdx.x >> 5;
    __shared__ float4 s_hi[8][CL], s_lo[8][CL];
    const int ncl = c.ncol * c.maxcl;
    const int cur = (int)((*s.step_base + step_off) & 1);
    const uint32_t below = (1u << lane) - 1u;
    for (int I = blockIdx.x * wpb + wl; I < ncl; I += gridDim.x * wpb) {
        __syncwarp();
        if (lane < CL) {
            // padding slots (no atom) are placed out of reach: their copies in
            // the buffer the step kernel writes are never refreshed
            const bool real = c.smol[I * CL + lane] >= 0;
            const float4 far = make_float4(1e30f, 1e30f, 1e30f, 0.f);
            s_hi[wl][lane] = real ? c.sphi[cur][I * CL + lane] : far;
            s_lo[wl][lane] = real ? c.splo[cur][I * CL + lane] : make_float4(0.f, 0.f, 0.f, 0.f);
            c.pref[I * CL + lane] = c.sphi[cur][I * CL + lane];
        }
        __syncwarp();
        for (int L = 0; L < c.nlists; ++L) {
            const int n = c.lcnt[L][I];
            const int* src = c.lst[L] + (size_t)I * c.capj[L];
            int* dst = c.plst[L] + (size_t)I * c.capj[L];
            int m = 0;
            const float R2 = c.prs2[L];
            // two passes of 32 entries per iteration: their loads are in flight together
            for (int e0 = 0; e0 < n; e0 += 64) {
                // (an entry's image code fills its top bits: validity comes from the index)
                const int ea = e0 + lane, eb = ea + 32;
                const bool va = ea < n, vb = eb < n;
                const int enta = va ? src[ea] : 0, entb = vb ? src[eb] : 0;
                const float4 ha = va ? c.sphi[cur][enta & 0x07FFFFFF] : make_float4(0.f, 0.f, 0.f, 0.f);
                const float4 hb = vb ? c.sphi[cur][entb & 0x07FFFFFF] : make_float4(0.f, 0.f, 0.f, 0.f);
                const bool ka = va && prune_keep(s, p, cur, enta, ha, s_hi[wl], s_lo[wl], R2);
                const bool kb = vb && prune_keep(s, p, cur, entb, hb, s_hi[wl], s_lo[wl], R2);
                const uint32_t ba = __ballot_sync(0xffffffffu, ka), bb = __ballot_sync(0xffffffffu, kb);
                if (ka) dst[m + __popc(ba & below)] = enta;
                m += __popc(ba);
                if (kb) dst[m + __popc(bb & below)] = entb;
                m += __popc(bb);
            }
            if (lane == 0) {
                c.pcnt[L][I] = m;
                // work items of I's pruned list, at slots taken from a counter
                // (their order does not matter: the sums are fixed point)
                const int nch = (m + EPW - 1) / EPW;
                const int b = nch ? atomicAdd(&c.pnitems[2 + L], nch) : 0;
                for (int k = 0; k < nch; ++k)
                    if (b + k < c.capitems) c.pitems[L][b + k] = make_int2(I, k * EPW);
            }
        }
    }
    if (!cl_last_cta(&c.done_ctr[2])) return;
    if (threadIdx.x < 2) {
        const int L = threadIdx.x;
        const int n = atomicExch(&c.pnitems[2 + L], 0);
        c.pnitems[L] = min(n, c.capitems);
        if (n > c.capitems) atomicOr(s.err, BERR_LIST_OVERFLOW);
    }
    if (threadIdx.x == 0) *c.prune = 0;
}

__device__ __forceinline__ void fix_add(unsigned long long* a, float v) {
    if (v != 0.f) atomicAdd(a, fix_round<32>(v));
}

// Exact FP64 cutoff test of one pair near r_c, out of line (rare).
__device__ __noinline__ bool cl_exact_inside(const DevSys& s, const Params& p, int cur, int a, int b) {
    return exact_r2(s, p, cur, a, b) < p.rc2_d;
}


// The pairs of one list entry (atom slot sj, split position hj/lj in the
// image of the entry) whose FP32 r^2 fell within the rounding band of r_c^2
// (bits of `near`): each takes the exact FP64 cutoff test; a pair inside
// adds its i side straight to the accumulator of its slot (rare) and its j
// side to the lane's sums.
template <int PART>
__device__ __forceinline__ void near_pairs(const DevSys& s, const Params& p, int cur, int I, int sj, float4 hj, float4 lj,
                                        uint32_t near, const float4* s_hi, const float4* s_lo, const float* s_c12,
                                        const float* s_c6, float& gjx, float& gjy, float& gjz, int& npair) {
    const DevClu& c = s.cl;
    const size_t ns = (size_t)c.ncol * c.maxcl * CL;
    for (; near; near &= near - 1u) {
        const int a = __ffs(near) - 1;
        if (!(exact_r2(s, p, cur, c.cl_atom[I * CL + a], c.cl_atom[sj]) < p.rc2_d)) continue;
        const float4 hi = s_hi[a], lo = s_lo[a];
        const float3 d = pair_disp(p, hi, lo, hj, lj);
        const float r2 = d.x * d.x + d.y * d.y + d.z * d.z;
        const int tp = type_of(lo) * BOUNCE_MAXT + type_of(lj);
        const float w = pairsum_w<PART>(p, r2, p.kcoul * hi.w * hj.w, s_c12[tp], s_c6[tp]);
        fix_add(c.acc + (size_t)I * CL + a, w * d.x);
        fix_add(c.acc + ns + (size_t)I * CL + a, w * d.y);
        fix_add(c.acc + 2 * ns + (size_t)I * CL + a, w * d.z);
        gjx = fmaf(-w, d.x, gjx);
        gjy = fmaf(-w, d.y, gjy);
        gjz = fmaf(-w, d.z, gjz);
        ++npair;
    }
}

// The 8 pairs of one list entry j (split position hj/lj in the entry's
// image, molecule mj, type tj, slot sj) with the atoms of cluster I (shared
// memory): i sides into gi, the j side into gj, in-cutoff pairs counted,
// pairs within the rounding band of r_c flagged in `near` for the exact
// test.  PER: minimum image per pair (clusters near half a box edge).
template <int PART, bool PER>
__device__ __forceinline__ void entry_pairs(const Params& p, const float4* shi, const float4* slo, const int* smol,
                                            const float* c12t, const float* c6t, float4 hj, float4 lj, int mj, int tj,
                                            int sj, int I, float (&gi)[CL][3], float& gjx, float& gjy, float& gjz,
                                            uint32_t& near, int& npair) {
#pragma unroll
    for (int a = 0; a < CL; ++a) {
        const float4 hi = shi[a], lo = slo[a];
        const int mi = smol[a];
        float3 d;
        if (PER) {
            d = pair_disp(p, hi, lo, hj, lj);
        } else {
            d.x = (hi.x - hj.x) + (lo.x - lj.x);
            d.y = (hi.y - hj.y) + (lo.y - lj.y);
            d.z = (hi.z - hj.z) + (lo.z - lj.z);
        }
        const float r2 = d.x * d.x + d.y * d.y + d.z * d.z;
        const bool ok = mi >= 0 && mi != mj && sj > I * CL + a;
        const bool in = ok && r2 < p.rc2_lo;
        near |= (ok && r2 >= p.rc2_lo && r2 <= p.rc2_hi) ? 1u << a : 0u;
        const int tp = type_of(lo) * BOUNCE_MAXT + tj;
        const float w0 = pairsum_w<PART>(p, in ? r2 : 1.f, p.kcoul * hi.w * hj.w, c12t[tp], c6t[tp]);
        const float wv = in ? w0 : 0.f;
        npair += in ? 1 : 0;
        gi[a][0] = fmaf(wv, d.x, gi[a][0]);
        gi[a][1] = fmaf(wv, d.y, gi[a][1]);
        gi[a][2] = fmaf(wv, d.z, gi[a][2]);
        gjx = fmaf(-wv, d.x, gjx);
        gjy = fmaf(-wv, d.y, gjy);
        gjz = fmaf(-wv, d.z, gjz);
    }
}

// Pair sums over the work items of list `L`.  PART 3: the F_0 share
// (1 - chi) W'_sw + W'_fixed; PART 5: the full W'.  A warp takes an item of
// cluster I: lanes hold one list atom j each, the 8 atoms of I are read from
// shared memory in turn; the j side of every pair is summed in the lane's
// registers and added once per item, the i side is kept per lane for the 8
// atoms and reduced over the warp at the end of the item.
template <int PART>
__global__ void __launch_bounds__(256, CL_PAIRS_MIN_CTAS) k_cl_pairs(DevSys s, Params p, int step_off, int L) {
    chain_enter();
    __shared__ float4 s_hi[8][CL], s_lo[8][CL];
    __shared__ int s_mol[8][CL];
    __shared__ float s_c12[BOUNCE_MAXT * BOUNCE_MAXT], s_c6[BOUNCE_MAXT * BOUNCE_MAXT];
    if (threadIdx.x < BOUNCE_MAXT * BOUNCE_MAXT) {
        s_c12[threadIdx.x] = p.c12[threadIdx.x];
        s_c6[threadIdx.x] = p.c6[threadIdx.x];
    }
    __syncthreads();
    const DevClu& c = s.cl;
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const int cur = (int)((*s.step_base + step_off) & 1);
    const int capj = c.capj[L];
    const int* lst = c.plst[L];
    const int* lcnt = c.pcnt[L];
    const int nit = c.pnitems[L];
    const size_t ns = (size_t)c.ncol * c.maxcl * CL;
    const float4* sphi = c.sphi[cur];
    const float4* splo = c.splo[cur];
    int npair = 0;
    // items are fetched from a counter, so that no warp idles while its
    // CTA's other warps still work (the items differ in length)
    for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(&c.pnitems[4 + L], 1);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= nit) break;
        const int2 w = c.pitems[L][it];
        const int I = w.x, e1 = min(w.y + EPW, lcnt[I]);
        __syncwarp();
        if (lane < CL) {
            s_hi[wl][lane] = sphi[I * CL + lane];
            s_lo[wl][lane] = splo[I * CL + lane];
            s_mol[wl][lane] = c.smol[I * CL + lane];
        }
        __syncwarp();
        float gi[CL][3];
#pragma unroll
        for (int a = 0; a < CL; ++a) gi[a][0] = gi[a][1] = gi[a][2] = 0.f;
        for (int e = w.y + lane; e < e1; e += 32) {
            const int ent = __ldg(lst + (size_t)I * capj + e);
            const int sj = ent & 0x07FFFFFF, code = (int)((uint32_t)ent >> 27);
            float4 hj = sphi[sj], lj = splo[sj];
            const int mj = c.smol[sj];
            const int tj = type_of(lj);
            if (code != NO_SHIFT && code != PER_PAIR) {
                const float kx = (float)(code / 9 - 1), ky = (float)((code / 3) % 3 - 1), kz = (float)(code % 3 - 1);
                shift_split(hj.x, lj.x, kx * p.Lhi[0], kx * p.Llo[0]);
                shift_split(hj.y, lj.y, ky * p.Lhi[1], ky * p.Llo[1]);
                shift_split(hj.z, lj.z, kz * p.Lhi[2], kz * p.Llo[2]);
            }
            float gjx = 0.f, gjy = 0.f, gjz = 0.f;
            uint32_t near = 0u;  // pairs within the FP32 rounding band of r_c
            // the rare per-pair minimum image takes its own copy of the loop,
            // so that the common one carries no minimum-image arithmetic
            if (code == PER_PAIR)
                entry_pairs<PART, true>(p, s_hi[wl], s_lo[wl], s_mol[wl], s_c12, s_c6, hj, lj, mj, tj, sj, I, gi, gjx,
                                        gjy, gjz, near, npair);
            else
                entry_pairs<PART, false>(p, s_hi[wl], s_lo[wl], s_mol[wl], s_c12, s_c6, hj, lj, mj, tj, sj, I, gi, gjx,
                                         gjy, gjz, near, npair);
            if (near) near_pairs<PART>(s, p, cur, I, sj, hj, lj, near, s_hi[wl], s_lo[wl], s_c12, s_c6, gjx, gjy, gjz,
                                       npair);
            fix_add(c.acc + sj, gjx);
            fix_add(c.acc + ns + sj, gjy);
            fix_add(c.acc + 2 * ns + sj, gjz);
        }
        // i side: each of the 24 sums over the warp; lane 3 a + d adds component d of atom a
        float mine = 0.f;
#pragma unroll
        for (int a = 0; a < CL; ++a)
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                float v = gi[a][d];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 3 * a + d) mine = v;
            }
        if (lane < 3 * CL && s_mol[wl][lane / 3] >= 0) fix_add(c.acc + (size_t)(lane % 3) * ns + I * CL + lane / 3, mine);
    }
    npair = warp_sum_i(npair);
    if (lane == 0 && npair) atomicAdd(&s.cnt[PART == 3 ? CNT_SHORT_PAIRS : CNT_FULL_PAIRS], (unsigned long long)npair);
    // every warp has seen the counter past the last item: the last CTA resets it
    if (cl_last_cta(&c.done_ctr[3]) && threadIdx.x == 0) c.pnitems[4 + L] = 0;
}

// The accumulated pair sums of every atom added to out (n x 3, FP64), and
// the accumulators cleared for the next evaluation.
__global__ void k_cl_collect(DevSys s, double* out) {
    const DevClu& c = s.cl;
    const size_t ns = (size_t)c.ncol * c.maxcl * CL;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < s.n; i += gridDim.x * blockDim.x) {
        const int sl = c.a2s[i];
        for (int d = 0; d < 3; ++d) {
            const long long v = (long long)c.acc[d * ns + sl];
            c.acc[d * ns + sl] = 0ull;
            out[3 * (size_t)i + d] += (double)v * CL_UNFIX;
        }
    }
}

}  // namespace

void launch_cluster_rebuild(const DevSys& s, const Params& p, int step_off, bool force, cudaStream_t st) {
    const int f = force ? 1 : 0;
    const int tb = 1024, gb = (s.n + tb - 1) / tb;
    launch_chained(k_cl_count, gb, tb, 0, st, s, p, step_off, f);
    launch_chained(k_cl_scatter, gb, tb, 0, st, s, p, step_off, f);
    launch_chained(k_cl_sort, std::min(s.cl.ncol, 152 * 8), SORT_NT, 0, st, s, p, step_off, f);
    const int ncl = s.cl.ncol * s.cl.maxcl;
    launch_chained(k_cl_search, std::min((ncl + 7) / 8, 152 * 8), 256, 0, st, s, p, step_off, f);
    launch_chained(k_cl_prune, std::min((ncl + 7) / 8, 152 * 8), 256, 0, st, s, p, step_off, f);
}

// CTAs of the pair kernel that fit on the GPU at once (the warps fetch their
// work items, so one resident wave covers any number of items)
template <int PART>
static int cl_pairs_grid() {
    static int blocks = 0;
    if (!blocks) {
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_cl_pairs<PART>, 256, 0);
        blocks = std::max(1, sms * std::max(per, 1));
    }
    return blocks;
}

void prepare_cluster_pairs() {
    cl_pairs_grid<3>();
    cl_pairs_grid<5>();
}

void launch_cluster_pairs(const DevSys& s, const Params& p, int step_off, int part, int list, cudaStream_t st) {
    if (part == 3) launch_chained(k_cl_pairs<3>, cl_pairs_grid<3>(), 256, 0, st, s, p, step_off, list);
    else launch_chained(k_cl_pairs<5>, cl_pairs_grid<5>(), 256, 0, st, s, p, step_off, list);
}

void launch_cluster_collect(const DevSys& s, double* out, cudaStream_t st) {
    k_cl_collect<<<(s.n + 255) / 256, 256, 0, st>>>(s, out);
}
