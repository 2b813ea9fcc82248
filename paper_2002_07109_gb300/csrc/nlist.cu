// Candidate rows of the jump step and the pair sums (paper Sec. V, first
// paragraph: the partner J of atom i is drawn uniformly among the particles
// interacting with i).  Row of atom i: every atom j of another molecule with
// r_ij^2 < r_list^2 (FP64, minimum image), in ascending j.
//
// GPU design: a cell grid of edge >= r_list / 3 (counting sort: count, scan,
// scatter), then one warp per atom scans the cells that meet its r_list
// sphere, screens each candidate in FP32 from the high position parts and
// settles the few candidates near r_list exactly in FP64.  Accepted
// candidates set a bit in a per-warp bitmap over all atom indices in shared
// memory (one per partner type with per-type-pair bounds, then a bitmap of
// the short-row members, r < r_off + skin);
// reading a bitmap back in word order yields the row already in ascending
// order (no sort), and duplicate visits of a cell are harmless.
// Every kernel returns at once unless a rebuild is pending (the step kernel
// raises the flag when an atom has moved more than skin/2 since the last
// build), so the sequence can sit in a captured CUDA graph.  Three launches:
// cell counts (the CTA finishing last scans them), scatter into cell order
// (indices, positions and molecule ids), rows (the CTA finishing last clears
// the flag).
#include <algorithm>

#include "common.cuh"

namespace {

constexpr int RANGE_MAX = 128;  // cell-row runs per atom (<= 2 (2*3+1)^2 = 98)
constexpr int ROWS_NT = 256;    // threads per CTA of the row builder

// Entry of a gated rebuild kernel: after its predecessor in the chain, is a
// rebuild due (or forced)?
__device__ __forceinline__ bool pending(const DevSys& s, int force) {
    chain_enter();
    return force || *s.rebuild;
}

__device__ __forceinline__ void cell_of(const DevSys& s, const Params& p, float4 hi, int& cx, int& cy, int& cz) {
    if (p.periodic) {
        cx = min(max((int)(hi.x * s.ihx), 0), s.ncx - 1);
        cy = min(max((int)(hi.y * s.ihy), 0), s.ncy - 1);
        cz = min(max((int)(hi.z * s.ihz), 0), s.ncz - 1);
    } else {
        cx = min(max((int)floorf((hi.x - s.ox) * s.ihx), 0), s.ncx - 1);
        cy = min(max((int)floorf((hi.y - s.oy) * s.ihy), 0), s.ncy - 1);
        cz = min(max((int)floorf((hi.z - s.oz) * s.ihz), 0), s.ncz - 1);
    }
}

// True in the one CTA of the grid that finishes last (all others have
// completed their global writes); that CTA resets the counter to zero.
__device__ bool last_cta(unsigned int* ctr) {
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

// Exclusive scan of the cell counts by one CTA; resets the counts to zero
// for the next rebuild.
__device__ void cells_scan(const DevSys& s) {
    __shared__ int warp_tot[32];
    __shared__ int carry;
    int nc = s.ncx * s.ncy * s.ncz;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nc; base += blockDim.x) {
        int c = base + threadIdx.x;
        int v = c < nc ? __ldcg(&s.cell_count[c]) : 0;  // written by other CTAs' atomics
        int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        int x = v;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_tot[w] = x;
        __syncthreads();
        if (w == 0) {
            int t = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            warp_tot[lane] = t;
        }
        __syncthreads();
        int excl = carry + (w > 0 ? warp_tot[w - 1] : 0) + x - v;
        if (c < nc) {
            s.cell_start[c] = excl;
            s.cell_fill[c] = excl;
            s.cell_count[c] = 0;
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) s.cell_start[nc] = carry;
}

// Cell counts; the CTA that finishes last scans them.
__global__ void k_cells_count(DevSys s, Params p, int step_off, int force) {
    if (!pending(s, force)) return;
    int cur = (int)((*s.step_base + step_off) & 1);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < s.n; i += gridDim.x * blockDim.x) {
        int cx, cy, cz;
        cell_of(s, p, s.phi[cur][i], cx, cy, cz);
        atomicAdd(&s.cell_count[(cz * s.ncy + cy) * s.ncx + cx], 1);
    }
    if (last_cta(&s.done_ctr[0])) cells_scan(s);
}

__global__ void k_cells_scatter(DevSys s, Params p, int step_off, int force) {
    if (!pending(s, force)) return;
    int cur = (int)((*s.step_base + step_off) & 1);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < s.n; i += gridDim.x * blockDim.x) {
        int cx, cy, cz;
        const float4 hi = s.phi[cur][i];
        cell_of(s, p, hi, cx, cy, cz);
        int pos = atomicAdd(&s.cell_fill[(cz * s.ncy + cy) * s.ncx + cx], 1);
        s.cell_atoms[pos] = i;
        s.cell_phi[pos] = hi;
        s.cell_mol[pos] = s.mol[i];
        s.cell_type[pos] = s.type[i];
    }
}

__device__ __forceinline__ bool in_list_fp64(const DevSys& s, const Params& p, int cur, int i, int j) {
    return exact_r2(s, p, cur, i, j) < p.rlist2_d;
}

// An FP32 minimum-image choice can differ from the FP64 one only when a
// component sits near half a box edge.
__device__ __forceinline__ bool image_ambiguous(const Params& p, float4 hi, float4 hj) {
    if (!p.periodic) return false;
    float fx = fabsf((hi.x - hj.x) * p.invL[0]), fy = fabsf((hi.y - hj.y) * p.invL[1]),
          fz = fabsf((hi.z - hj.z) * p.invL[2]);
    fx -= floorf(fx);
    fy -= floorf(fy);
    fz -= floorf(fz);
    return fabsf(fx - 0.5f) < 1e-4f || fabsf(fy - 0.5f) < 1e-4f || fabsf(fz - 0.5f) < 1e-4f;
}

// Candidate runs of atom i (one warp): up to two contiguous runs of cells
// per (z, y) cell row meeting the r_list sphere (periodic wrap), each a
// contiguous run of atoms in the cell-sorted arrays; rb / rl / rp receive
// their starts, lengths and exclusive prefix, the return value is the number
// of candidates and nr the number of runs.
__device__ int candidate_runs(const DevSys& s, const Params& p, float4 hi, int* rb, int* rl, int* rp, int& nr) {
    const int lane = threadIdx.x & 31;
    // unclamped cell coordinates of atom i
    const float fx = p.periodic ? hi.x * s.ihx : (hi.x - s.ox) * s.ihx;
    const float fy = p.periodic ? hi.y * s.ihy : (hi.y - s.oy) * s.ihy;
    const float fz = p.periodic ? hi.z * s.ihz : (hi.z - s.oz) * s.ihz;
    int cx, cy, cz;
    cell_of(s, p, hi, cx, cy, cz);
    // geometric culling is valid unless atom i sits outside a droplet grid
    const bool cull = p.periodic || (fx >= 0.f && fy >= 0.f && fz >= 0.f && fx < (float)s.ncx &&
                                     fy < (float)s.ncy && fz < (float)s.ncz);
    const float rc2 = p.rcull * p.rcull;
    // axes narrower than the stencil are scanned once, without culling or wrap
    const bool fullz = s.ncz <= 2 * s.mz + 1, fully = s.ncy <= 2 * s.my + 1, fullx = s.ncx <= 2 * s.mx + 1;
    const int z0 = fullz ? 0 : cz - s.mz, z1 = fullz ? s.ncz - 1 : cz + s.mz;
    const int y0 = fully ? 0 : cy - s.my, y1 = fully ? s.ncy - 1 : cy + s.my;
    // 1) lanes compute the candidate ranges of all (z, y) cell rows in
    //    parallel: up to two contiguous runs of cells per row (periodic
    //    wrap), each a contiguous run of atoms in the cell-sorted array
    const int nzr = z1 - z0 + 1, nyr = y1 - y0 + 1, nrows = nzr * nyr;
    int nr_tot = 0;
    for (int r0 = 0; r0 < nrows; r0 += 32) {
        const int r = r0 + lane;
        int b0 = 0, l0 = 0, b1 = 0, l1 = 0;
        if (r < nrows) {
            const int zu = z0 + r / nyr, yu = y0 + r % nyr;
            int zz = zu, yy = yu;
            bool ok = true;
            if (!fullz) {
                if (p.periodic) zz = (zu % s.ncz + s.ncz) % s.ncz;
                else ok = zu >= 0 && zu < s.ncz;
            }
            if (!fully) {
                if (p.periodic) yy = (yu % s.ncy + s.ncy) % s.ncy;
                else ok = ok && yu >= 0 && yu < s.ncy;
            }
            float gz = 0.f, gy = 0.f;
            if (cull && !fullz) gz = fmaxf(fmaxf((float)zu - fz, fz - (float)(zu + 1)), 0.f) * s.hz;
            if (cull && !fully) gy = fmaxf(fmaxf((float)yu - fy, fy - (float)(yu + 1)), 0.f) * s.hy;
            const float g2 = gz * gz + gy * gy;
            if (ok && g2 <= rc2) {
                int xa, xb;
                if (fullx) {
                    xa = 0;
                    xb = s.ncx - 1;
                } else if (cull) {
                    const float hw = sqrtf(rc2 - g2) * s.ihx;
                    xa = max((int)floorf(fx - hw), cx - s.mx);
                    xb = min((int)floorf(fx + hw), cx + s.mx);
                } else {
                    xa = cx - s.mx;
                    xb = cx + s.mx;
                }
                const int rowc = (zz * s.ncy + yy) * s.ncx;
                int ca[3], cb[3], nrr = 0;
                if (fullx) {
                    ca[0] = xa; cb[0] = xb; nrr = 1;
                } else if (p.periodic) {
                    if (xa < 0) { ca[nrr] = xa + s.ncx; cb[nrr] = s.ncx - 1; ++nrr; xa = 0; }
                    if (xb >= s.ncx) { ca[nrr] = 0; cb[nrr] = xb - s.ncx; ++nrr; xb = s.ncx - 1; }
                    if (xa <= xb) { ca[nrr] = xa; cb[nrr] = xb; ++nrr; }
                } else {
                    xa = max(xa, 0);
                    xb = min(xb, s.ncx - 1);
                    if (xa <= xb) { ca[0] = xa; cb[0] = xb; nrr = 1; }
                }
                if (nrr > 0) {
                    b0 = s.cell_start[rowc + ca[0]];
                    l0 = s.cell_start[rowc + cb[0] + 1] - b0;
                }
                if (nrr > 1) {
                    b1 = s.cell_start[rowc + ca[1]];
                    l1 = s.cell_start[rowc + cb[1] + 1] - b1;
                }
                if (nrr > 2) {  // both wraps: the span covers the whole row
                    b0 = s.cell_start[rowc];
                    l0 = s.cell_start[rowc + s.ncx] - b0;
                    l1 = 0;
                }
            }
        }
        // compact non-empty runs into the per-warp list, in row order
        const bool h0 = l0 > 0, h1 = l1 > 0;
        const int cnt = (int)h0 + (int)h1;
        int x = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        int pos = nr_tot + x - cnt;
        if (h0 && pos < RANGE_MAX) { rb[pos] = b0; rl[pos] = l0; ++pos; }
        if (h1 && pos < RANGE_MAX) { rb[pos] = b1; rl[pos] = l1; }
        nr_tot += __shfl_sync(0xffffffffu, x, 31);
    }
    nr_tot = min(nr_tot, RANGE_MAX);
    __syncwarp();
    // 2) exclusive prefix of the run lengths
    int total_c = 0;
    for (int r0 = 0; r0 < nr_tot; r0 += 32) {
        const int r = r0 + lane;
        const int len = r < nr_tot ? rl[r] : 0;
        int x = len;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (r < nr_tot) rp[r] = total_c + x - len;
        total_c += __shfl_sync(0xffffffffu, x, 31);
    }
    __syncwarp();
    nr = nr_tot;
    return total_c;
}

// Writes the set bits of a warp's bitmap, in ascending order, as indices to
// row[0 .. cap) and returns their count (which may exceed cap; cap may be
// zero or negative, then nothing is written).  Passes of 32 words: a prefix
// of their popcounts, then the pass's set bits are spread over the lanes,
// 32 at a time: output k of the pass finds its word by a shuffle search over
// the prefix and its bit by a popcount halving search, so the stores are
// contiguous and the cost
// follows the number of set bits, not of non-empty words.  Empty passes cost
// one load and a vote.
// Position of the set bit of rank r (0-based, r < popc(b)) in b.
__device__ __forceinline__ int select_bit(uint32_t b, int r) {
    int pos = 0;
#pragma unroll
    for (int half = 16; half > 0; half >>= 1) {
        const int c = __popc(b & ((1u << half) - 1u));
        if (r >= c) {
            r -= c;
            b >>= half;
            pos += half;
        }
    }
    return pos;
}

__device__ int expand_bitmap(const uint32_t* bm, int nwords, int* row, int cap) {
    const int lane = threadIdx.x & 31;
    int total = 0;
    for (int w0 = 0; w0 < nwords; w0 += 32) {
        const int w = w0 + lane;
        const uint32_t bits = w < nwords ? bm[w] : 0u;
        if (!__any_sync(0xffffffffu, bits != 0u)) continue;
        const int c = __popc(bits);
        int x = c;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        const int excl = x - c;  // set bits of this pass before word w
        const int tc = __shfl_sync(0xffffffffu, x, 31);
        for (int k0 = 0; k0 < tc; k0 += 32) {
            const int k = k0 + lane;
            // last lane l with excl_l <= k (the words of lanes before it hold fewer than k + 1 bits)
            int l = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const int e = __shfl_sync(0xffffffffu, excl, l + step);
                if (e <= k) l += step;
            }
            const uint32_t b = __shfl_sync(0xffffffffu, bits, l);
            const int r = k - __shfl_sync(0xffffffffu, excl, l);
            if (k < tc) {
                const int pos = total + k;
                if (pos < cap) row[pos] = ((w0 + l) << 5) + select_bit(b, r);
            }
        }
        total += tc;
    }
    return total;
}

// Rows of the cell-list builder, one warp per atom (systems whose bitmaps
// over all atoms are small): the warp screens the candidates of its atom and
// sets bits in its own bitmaps, then reads them back in word order.
__global__ void k_rows_warp(DevSys s, Params p, int step_off, int force, int words_per_warp) {
    if (!pending(s, force)) return;
    extern __shared__ uint32_t smem_bm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const int nwords = (s.n + 31) >> 5;
    // long-row bitmaps (one per partner type with per-type-pair bounds), then
    // the short-row bitmap
    const int wr = (nwords + 3) & ~3, nbm = p.typed ? p.n_types : 1;
    uint32_t* bm = smem_bm + (size_t)warp * words_per_warp;
    uint32_t* bs = bm + (size_t)nbm * wr;
    const int cur = (int)((*s.step_base + step_off) & 1);
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&s.cnt[CNT_REBUILDS], 1ull);
    for (int i = blockIdx.x * wpb + warp; i < s.n; i += gridDim.x * wpb) {
        for (int w = lane; w < (nbm + 1) * wr; w += 32) bm[w] = 0u;
        __syncwarp();
        const float4 hi = s.phi[cur][i];
        const int mi = s.mol[i];
        int* rb = (int*)(bm + words_per_warp - 3 * RANGE_MAX);
        int* rl = rb + RANGE_MAX;
        int* rp = rl + RANGE_MAX;
        int nr_tot;
        const int total_c = candidate_runs(s, p, hi, rb, rl, rp, nr_tot);
        __syncwarp();
        // 3) all lanes stride over the concatenated candidates (cell-ordered
        //    copies: consecutive lanes read consecutive entries of a run)
        int lo_r = 0;  // run of candidate t: rp[lo_r] <= t < rp[lo_r + 1]; t only grows
        for (int t = lane; t < total_c; t += 32) {
            while (lo_r + 1 < nr_tot && rp[lo_r + 1] <= t) ++lo_r;
            const int idx = rb[lo_r] + (t - rp[lo_r]);
            const int j = s.cell_atoms[idx];
            const int mj = s.cell_mol[idx];
            // screen with the high FP32 parts; the band covers their error
            const float4 hj = s.cell_phi[idx];
            if (j == i || mj == mi) continue;
            float dx = hi.x - hj.x, dy = hi.y - hj.y, dz = hi.z - hj.z;
            if (p.periodic) {
                dx -= rintf(dx * p.invL[0]) * p.Lhi[0];
                dy -= rintf(dy * p.invL[1]) * p.Lhi[1];
                dz -= rintf(dz * p.invL[2]) * p.Lhi[2];
            }
            const float r2 = dx * dx + dy * dy + dz * dz;
            bool in;
            if (r2 < p.rlist2_lo && !image_ambiguous(p, hi, hj)) in = true;
            else if (r2 > p.rlist2_hi && !image_ambiguous(p, hi, hj)) in = false;
            else in = in_list_fp64(s, p, cur, i, j);
            if (in) {
                uint32_t* bt = p.typed ? bm + (size_t)s.cell_type[idx] * wr : bm;
                atomicOr(&bt[j >> 5], 1u << (j & 31));
                // short rows: r < r_off + skin (rshort2 carries a 1e-4 margin)
                if (r2 < p.rshort2) atomicOr(&bs[j >> 5], 1u << (j & 31));
            }
        }
        __syncwarp();
        // bitmaps -> ascending rows
        // (typed rows: the type groups one after the other, group sizes to nseg)
        int total = 0;
        for (int t = 0; t < nbm; ++t) {
            const int c = expand_bitmap(bm + (size_t)t * wr, nwords, s.rows + (size_t)i * s.cap + total,
                                        s.cap - total);
            if (p.typed && lane == 0) s.nseg[(size_t)i * BOUNCE_MAXT + t] = c;
            total += c;
        }
        const int ns = p.rshort2 < INFINITY ? expand_bitmap(bs, nwords, s.srows + (size_t)i * s.caps, s.caps) : 0;
        if (lane == 0) {
            s.nlong[i] = min(total, s.cap);
            if (total > s.cap) atomicOr(s.err, BERR_LIST_OVERFLOW);
            s.nshort[i] = min(ns, s.caps);
            if (ns > s.caps) atomicOr(s.err, BERR_SHORT_OVERFLOW);
            s.refx[i] = s.qx[cur][i];
            s.refy[i] = s.qy[cur][i];
            s.refz[i] = s.qz[cur][i];
        }
        __syncwarp();
    }
    if (last_cta(&s.done_ctr[1])) *s.rebuild = 0;
}

// Rows of the cell-list builder for large systems, one CTA per atom: warp 0
// finds the candidate runs, all threads screen the candidates and set bits in
// the CTA's bitmaps (one per partner type with per-type-pair bounds, one for
// the short rows) and a touched flag per 32-word group; then the touched
// groups in order, their popcounts and prefix, and the warps expand them into
// the rows in ascending index and clear them.  The work per atom follows its
// neighbours, not n, and the bitmaps are shared by the CTA's 8 warps.
__global__ void __launch_bounds__(ROWS_NT) k_rows_cta(DevSys s, Params p, int step_off, int force) {
    if (!pending(s, force)) return;
    extern __shared__ uint32_t smem_bm[];
    __shared__ int s_nr, s_tc, s_ntg, s_tot[BOUNCE_MAXT + 1];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = ROWS_NT / 32;
    const int nwords = (s.n + 31) >> 5, wr = (nwords + 3) & ~3, nbm = p.typed ? p.n_types : 1;
    // short rows exist only for a finite short radius (else F_0 reads the
    // long rows and srows has a single slot)
    const bool has_short = p.rshort2 < INFINITY;
    const int nb = nbm + (has_short ? 1 : 0);  // bitmaps in use
    const int ngroups = (nwords + 31) >> 5;
    uint32_t* bm = smem_bm;  // bitmaps b = 0 .. nbm - 1 (long rows), b = nbm (short rows)
    uint8_t* touched = (uint8_t*)(bm + (size_t)(nbm + 1) * wr);
    int* goff = (int*)(touched + ((ngroups + 15) & ~15));  // per (bitmap, touched group): count, then offset
    int* tg = goff + (((nbm + 1) * ngroups + 3) & ~3);     // touched groups, ascending
    int* rb = tg + ((ngroups + 3) & ~3);
    int* rl = rb + RANGE_MAX;
    int* rp = rl + RANGE_MAX;
    const int cur = (int)((*s.step_base + step_off) & 1);
    if (blockIdx.x == 0 && tid == 0) atomicAdd(&s.cnt[CNT_REBUILDS], 1ull);
    // full clear once; after each atom only its touched groups are cleared
    for (int w = tid; w < (nbm + 1) * wr; w += ROWS_NT) bm[w] = 0u;
    for (int g = tid; g < ngroups; g += ROWS_NT) touched[g] = 0;
    __syncthreads();
    for (int i = blockIdx.x; i < s.n; i += gridDim.x) {
        const float4 hi = s.phi[cur][i];
        const int mi = s.mol[i];
        if (warp == 0) {
            int nr;
            const int tc = candidate_runs(s, p, hi, rb, rl, rp, nr);
            if (lane == 0) {
                s_nr = nr;
                s_tc = tc;
            }
        }
        __syncthreads();
        // screen the candidates (each thread's t only grows, so its run index
        // advances monotonically)
        const int nr = s_nr, tc = s_tc;
        int lo_r = 0;
        for (int t = tid; t < tc; t += ROWS_NT) {
            while (lo_r + 1 < nr && rp[lo_r + 1] <= t) ++lo_r;
            const int idx = rb[lo_r] + (t - rp[lo_r]);
            const int j = s.cell_atoms[idx];
            const int mj = s.cell_mol[idx];
            // screen with the high FP32 parts; the band covers their error
            const float4 hj = s.cell_phi[idx];
            if (j == i || mj == mi) continue;
            float dx = hi.x - hj.x, dy = hi.y - hj.y, dz = hi.z - hj.z;
            if (p.periodic) {
                dx -= rintf(dx * p.invL[0]) * p.Lhi[0];
                dy -= rintf(dy * p.invL[1]) * p.Lhi[1];
                dz -= rintf(dz * p.invL[2]) * p.Lhi[2];
            }
            const float r2 = dx * dx + dy * dy + dz * dz;
            bool in;
            if (r2 < p.rlist2_lo && !image_ambiguous(p, hi, hj)) in = true;
            else if (r2 > p.rlist2_hi && !image_ambiguous(p, hi, hj)) in = false;
            else in = in_list_fp64(s, p, cur, i, j);
            if (in) {
                uint32_t* bt = p.typed ? bm + (size_t)s.cell_type[idx] * wr : bm;
                atomicOr(&bt[j >> 5], 1u << (j & 31));
                touched[j >> 10] = 1;  // every thread writes the same value: no atomic needed
                // short rows: r < r_off + skin (rshort2 carries a 1e-4 margin)
                if (has_short && r2 < p.rshort2) atomicOr(&bm[(size_t)nbm * wr + (j >> 5)], 1u << (j & 31));
            }
        }
        __syncthreads();
        // the touched groups, ascending (warp 0)
        if (warp == 0) {
            int k = 0;
            for (int g0 = 0; g0 < ngroups; g0 += 32) {
                const int g = g0 + lane;
                const bool t = g < ngroups && touched[g];
                const uint32_t m = __ballot_sync(0xffffffffu, t);
                if (t) tg[k + __popc(m & ((1u << lane) - 1u))] = g;
                k += __popc(m);
            }
            if (lane == 0) s_ntg = k;
        }
        __syncthreads();
        const int ntg = s_ntg, nitems = nb * ntg;
        // members per (bitmap, touched group)
        for (int it = warp; it < nitems; it += nwarp) {
            const int b = it / ntg, g = tg[it - b * ntg];
            const int w = (g << 5) + lane;
            const int c = warp_sum_i(w < nwords ? __popc(bm[(size_t)b * wr + w]) : 0);
            if (lane == 0) goff[it] = c;
        }
        __syncthreads();
        // exclusive prefix: the long bitmaps one after the other (typed rows:
        // type groups in order), the short bitmap on its own
        if (warp == 0) {
            int run = 0;
            for (int b = 0; b < nb; ++b) {
                if (b == nbm) run = 0;
                int tb = 0;
                for (int k0 = 0; k0 < ntg; k0 += 32) {
                    const int k = k0 + lane;
                    const int c = k < ntg ? goff[b * ntg + k] : 0;
                    int x = c;
                    for (int o = 1; o < 32; o <<= 1) {
                        const int y = __shfl_up_sync(0xffffffffu, x, o);
                        if (lane >= o) x += y;
                    }
                    if (k < ntg) goff[b * ntg + k] = run + tb + x - c;
                    tb += __shfl_sync(0xffffffffu, x, 31);
                }
                if (lane == 0) s_tot[b] = tb;
                run += tb;
            }
        }
        __syncthreads();
        // expand: lane w of the warp owns word w of the group; then clear it
        int* row = s.rows + (size_t)i * s.cap;
        int* srow = s.srows + (size_t)i * s.caps;
        for (int it = warp; it < nitems; it += nwarp) {
            const int b = it / ntg, g = tg[it - b * ntg];
            const int w = (g << 5) + lane;
            const uint32_t bits = w < nwords ? bm[(size_t)b * wr + w] : 0u;
            const int c = __popc(bits);
            int x = c;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            // the group's T set bits spread over the lanes: bit k lies in the
            // last word whose exclusive prefix is <= k (a shuffle binary
            // search), at its (k - prefix)-th set bit (a popcount descent)
            const int pre = x - c, T = __shfl_sync(0xffffffffu, x, 31), base = goff[it];
            int* out = b < nbm ? row : srow;
            const int cap = b < nbm ? s.cap : s.caps;
            for (int k0 = 0; k0 < T; k0 += 32) {
                const int k = k0 + lane;
                int src = 0;
#pragma unroll
                for (int h = 16; h > 0; h >>= 1) {
                    const int pc = __shfl_sync(0xffffffffu, pre, src + h);
                    if (pc <= k) src += h;
                }
                uint32_t v = __shfl_sync(0xffffffffu, bits, src);
                int r = k - __shfl_sync(0xffffffffu, pre, src), pos = 0;
#pragma unroll
                for (int h = 16; h >= 1; h >>= 1) {
                    const int lowc = __popc(v & ((1u << h) - 1u));
                    if (r >= lowc) {
                        r -= lowc;
                        v >>= h;
                        pos += h;
                    }
                }
                if (k < T && base + k < cap) out[base + k] = (((g << 5) + src) << 5) + pos;
            }
            if (w < nwords) bm[(size_t)b * wr + w] = 0u;
        }
        if (tid == 0) {
            int total = 0;
            for (int b = 0; b < nbm; ++b) {
                if (p.typed) s.nseg[(size_t)i * BOUNCE_MAXT + b] = s_tot[b];
                total += s_tot[b];
            }
            const int ns = has_short ? s_tot[nbm] : 0;
            s.nlong[i] = min(total, s.cap);
            if (total > s.cap) atomicOr(s.err, BERR_LIST_OVERFLOW);
            s.nshort[i] = min(ns, s.caps);
            if (ns > s.caps) atomicOr(s.err, BERR_SHORT_OVERFLOW);
            s.refx[i] = s.qx[cur][i];
            s.refy[i] = s.qy[cur][i];
            s.refz[i] = s.qz[cur][i];
        }
        for (int k = tid; k < ntg; k += ROWS_NT) touched[tg[k]] = 0;
        __syncthreads();
    }
    if (last_cta(&s.done_ctr[1])) *s.rebuild = 0;
}

// Rows of a batch of independent all-pairs replicas: every atom of the same
// replica outside the own molecule, ascending (no distance test: replicas
// have no cutoff), then the short rows and reference positions as above.
__global__ void k_rows_batch(DevSys s, Params p, int step_off, int force) {
    if (!pending(s, force)) return;
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    const int cur = (int)((*s.step_base + step_off) & 1);
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&s.cnt[CNT_REBUILDS], 1ull);
    for (int i = blockIdx.x * wpb + (threadIdx.x >> 5); i < s.n; i += gridDim.x * wpb) {
        const int r = s.rep_of[i], b = s.rep_off[r], e = s.rep_off[r + 1], mi = s.mol[i];
        int* row = s.rows + (size_t)i * s.cap;
        int total = 0;
        const int ngroups = p.typed ? p.n_types : 1;
        for (int tb = 0; tb < ngroups; ++tb) {  // typed rows: one pass per partner type
            const int before = total;
            for (int j0 = b; j0 < e; j0 += 32) {
                const int j = j0 + lane;
                const bool keep = j < e && s.mol[j] != mi && (!p.typed || s.type[j] == tb);
                const uint32_t m = __ballot_sync(0xffffffffu, keep);
                const int pos = total + __popc(m & ((1u << lane) - 1u));
                if (keep && pos < s.cap) row[pos] = j;
                total += __popc(m);
            }
            if (p.typed && lane == 0) s.nseg[(size_t)i * BOUNCE_MAXT + tb] = total - before;
        }
        __syncwarp();
        // short rows: ascending over the replica with the same high-part
        // screen as the cell-list builder (independent of the long row's order)
        const float4 hi = s.phi[cur][i];
        const int nl = min(total, s.cap);
        int ns = 0;
        int* srow = s.srows + (size_t)i * s.caps;
        for (int j0 = b; p.rshort2 < INFINITY && j0 < e; j0 += 32) {
            const int j = j0 + lane;
            bool keep = false;
            if (j < e && s.mol[j] != mi) {
                const float4 hj = s.phi[cur][j];
                const float dx = hi.x - hj.x, dy = hi.y - hj.y, dz = hi.z - hj.z;
                keep = dx * dx + dy * dy + dz * dz < p.rshort2;
            }
            const uint32_t m = __ballot_sync(0xffffffffu, keep);
            if (keep) {
                const int pos = ns + __popc(m & ((1u << lane) - 1u));
                if (pos < s.caps) srow[pos] = j;
            }
            ns += __popc(m);
        }
        if (lane == 0) {
            s.nlong[i] = nl;
            if (total > s.cap) atomicOr(s.err, BERR_LIST_OVERFLOW);
            s.nshort[i] = min(ns, s.caps);
            if (ns > s.caps) atomicOr(s.err, BERR_SHORT_OVERFLOW);
            s.refx[i] = s.qx[cur][i];
            s.refy[i] = s.qy[cur][i];
            s.refz[i] = s.qz[cur][i];
        }
        __syncwarp();
    }
    if (last_cta(&s.done_ctr[1])) *s.rebuild = 0;
}

__global__ void k_flag_moved(DevSys s, Params p, int cur) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < s.n; i += gridDim.x * blockDim.x) {
        const double ex = s.qx[cur][i] - s.refx[i], ey = s.qy[cur][i] - s.refy[i], ez = s.qz[cur][i] - s.refz[i];
        if (ex * ex + ey * ey + ez * ez > p.skin_half2) atomicOr(s.rebuild, 1);
    }
}

}  // namespace

void launch_flag_moved(const DevSys& s, const Params& p, int cur, cudaStream_t st) {
    k_flag_moved<<<(s.n + 255) / 256, 256, 0, st>>>(s, p, cur);
}

void launch_rebuild(const DevSys& s, const Params& p, int step_off, bool force, int bitmap_warps, size_t bitmap_bytes,
                    cudaStream_t st) {
    const int f = force ? 1 : 0;
    if (s.rep_of) {
        const int wpb = 8;
        launch_chained(k_rows_batch, (s.n + wpb - 1) / wpb, wpb * 32, 0, st, s, p, step_off, f);
        return;
    }
    const int tb = 1024;
    const int gb = (s.n + tb - 1) / tb;
    launch_chained(k_cells_count, gb, tb, 0, st, s, p, step_off, f);
    launch_chained(k_cells_scatter, gb, tb, 0, st, s, p, step_off, f);
    if (bitmap_warps > 0) {  // warp per atom, a grid-stride loop over one wave of CTAs
        const int words = (int)(bitmap_bytes / 4 / bitmap_warps);
        const int per_sm = std::max(1, std::min(8, (int)((227u << 10) / std::max<size_t>(bitmap_bytes, 1))));
        const int blocks = std::min((s.n + bitmap_warps - 1) / bitmap_warps, 152 * per_sm);
        launch_chained(k_rows_warp, blocks, bitmap_warps * 32, bitmap_bytes, st, s, p, step_off, f, words);
    } else {  // CTA per atom, a grid-stride loop over a GPU-filling grid (an idle launch stays small)
        const int blocks = std::min(s.n, 152 * 8);
        launch_chained(k_rows_cta, blocks, ROWS_NT, bitmap_bytes, st, s, p, step_off, f);
    }
}

void nlist_set_smem_limit(size_t bytes) {
    cudaFuncSetAttribute(k_rows_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    cudaFuncSetAttribute(k_rows_cta, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}
