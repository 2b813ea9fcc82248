// Candidate rows of the jump step and the pair sums (paper Sec. V, first
// paragraph: the partner J of atom i is drawn uniformly among the particles
// interacting with i).  Row of atom i: every atom j of another molecule with
// r_ij^2 < r_list^2 (FP64, minimum image), in ascending j.
//
// GPU design: a cell grid of edge >= r_list / 3 (counting sort: count, scan,
// scatter), then one warp per atom scans the cells that meet its r_list
// sphere, screens each candidate in FP32 from the high position parts and
// settles the few candidates near r_list exactly in FP64.  Accepted
// candidates set a bit in a per-warp bitmap over a window of atom indices
// centred on the atom's own (one per partner type with per-type-pair
// bounds, then a bitmap of the short-row members, r < r_off + skin);
// reading a bitmap back in word order yields the row already in ascending
// order (no sort), and duplicate visits of a cell are harmless.  Members
// outside the window take further passes (rare when atoms are numbered in
// spatial order).
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
// Atom i goes into the cells (ROWS_FILTER: only the types some jump row can hold).
__device__ __forceinline__ bool in_cells(const DevSys& s, const Params& p, int mode, int i) {
    return !(mode & ROWS_FILTER) || ((p.jcells >> s.type[i]) & 1);
}

__global__ void k_cells_count(DevSys s, Params p, int step_off, int force, int mode) {
    if (!pending(s, force)) return;
    int cur = (int)((*s.step_base + step_off) & 1);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < s.n; i += gridDim.x * blockDim.x) {
        if (!in_cells(s, p, mode, i)) continue;
        int cx, cy, cz;
        cell_of(s, p, s.phi[cur][i], cx, cy, cz);
        atomicAdd(&s.cell_count[(cz * s.ncy + cy) * s.ncx + cx], 1);
    }
    if (last_cta(&s.done_ctr[0])) cells_scan(s);
}

__global__ void k_cells_scatter(DevSys s, Params p, int step_off, int force, int mode) {
    if (!pending(s, force)) return;
    int cur = (int)((*s.step_base + step_off) & 1);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < s.n; i += gridDim.x * blockDim.x) {
        if (!in_cells(s, p, mode, i)) continue;
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
// zero or negative, then nothing is written); word w of the bitmap stands
// for atoms 32 (wbase + w) .. 32 (wbase + w) + 31.  Passes of 32 words: a prefix
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

__device__ int expand_bitmap(const uint32_t* bm, int nwords, int* row, int cap, int wbase = 0) {
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
                if (pos < cap) row[pos] = ((wbase + w0 + l) << 5) + select_bit(b, r);
            }
        }
        total += tc;
    }
    return total;
}

// Member test of candidate j for atom i at r_list: FP32 screen on the high
// parts, settled in FP64 inside the band around r_list or when the minimum
// image is ambiguous in FP32.  r2 receives the FP32 distance squared.
__device__ __forceinline__ bool row_member(const DevSys& s, const Params& p, int cur, int i, float4 hi, float4 hj,
                                           int j, float& r2) {
    float dx = hi.x - hj.x, dy = hi.y - hj.y, dz = hi.z - hj.z;
    if (p.periodic) {
        dx -= rintf(dx * p.invL[0]) * p.Lhi[0];
        dy -= rintf(dy * p.invL[1]) * p.Lhi[1];
        dz -= rintf(dz * p.invL[2]) * p.Lhi[2];
    }
    r2 = dx * dx + dy * dy + dz * dz;
    if (r2 < p.rlist2_lo && !image_ambiguous(p, hi, hj)) return true;
    if (r2 > p.rlist2_hi && !image_ambiguous(p, hi, hj)) return false;
    return in_list_fp64(s, p, cur, i, j);
}

// Rows of the cell-list builder, one warp per atom.  The warp's bitmaps (one
// per partner type with per-type-pair bounds, and one for the short rows)
// cover a window of `ww` words of atom indices centred on the atom's own
// index: reading them back in word order yields the row in ascending order
// without a sort.  The first pass screens the candidates, sets the bits of
// the members inside the window and counts, per type, the members below and
// above it; the window's members go to their final place in the row at
// once.  Members outside the window (index order far from spatial order)
// take further passes over windows below, then above it, each screening the
// candidates again; systems numbered in spatial order need one pass, and a
// window that spans every atom always does.
// mode: ROWS_ALL builds every row; ROWS_ACTIVE leaves the rows of atoms
// whose type has L* = 0 empty (they never propose: valid while the pair sums
// run over clusters or tiles and no short rows exist); ROWS_IDLE builds only
// those rows, at the current positions, keeping the reference positions and
// the rebuild flag of the last build (completing ROWS_ACTIVE rows for the
// energy, histogram and gradient entry points, which read every row);
// ROWS_READER builds every row the same way, into the readers' own row
// buffers.  ROWS_FILTER (with ROWS_ALL or ROWS_ACTIVE): the rows of the
// jump step keep only the partner types of the row's atom (Params::jpart),
// and the cells hold only the types some row can hold.
__global__ void k_rows_warp(DevSys s, Params p, int step_off, int force, int ww, int mode_in) {
    if (!pending(s, force)) return;
    extern __shared__ uint32_t smem_bm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const int nwords = (s.n + 31) >> 5;
    const int nbm = p.typed ? p.n_types : 1;
    const bool has_short = p.rshort2 < INFINITY;  // only when one window spans every atom
    const int nb = nbm + (has_short ? 1 : 0);
    const int per_warp = nb * ww + 3 * RANGE_MAX;
    uint32_t* bm = smem_bm + (size_t)warp * per_warp;
    uint32_t* bs = bm + (size_t)nbm * ww;  // the short-row bitmap (has_short)
    int* rb = (int*)(bm + (size_t)nb * ww);
    int* rl = rb + RANGE_MAX;
    int* rp = rl + RANGE_MAX;
    const int cur = (int)((*s.step_base + step_off) & 1);
    const int mode = mode_in & 7;
    const bool filt = (mode_in & ROWS_FILTER) != 0;
    // ROWS_IDLE and ROWS_READER builds leave the reference positions, the
    // rebuild flag and the rebuild count to the run's own builds
    const bool own = mode != ROWS_IDLE && mode != ROWS_READER;
    if (blockIdx.x == 0 && threadIdx.x == 0 && own) atomicAdd(&s.cnt[CNT_REBUILDS], 1ull);
    // the bitmaps start clear; after each atom only the words it touched are cleared
    for (int w = lane; w < nb * ww; w += 32) bm[w] = 0u;
    __syncwarp();
    // When the pair sums run over clusters or tiles, the rows serve only the
    // jump step, and an atom whose type has the bound L* = 0 never proposes
    // (its Poisson mean is 0).  act_order lists the atoms that can propose,
    // then the others: ROWS_ACTIVE builds the rows of the first n_act (the
    // others get empty rows and their reference positions), ROWS_IDLE the
    // rows of the rest; the warps stride over the listed atoms only, so the
    // work stays balanced whatever the order of the atom types.
    const bool split =
        mode != ROWS_ALL && mode != ROWS_READER && (s.cl.on || s.tl.on) && !has_short && s.act_order != nullptr;
    const int t0 = split && mode == ROWS_IDLE ? s.n_act : 0;
    const int t1 = split && mode == ROWS_ACTIVE ? s.n_act : s.n;
    if (split && mode == ROWS_ACTIVE)
        for (int t = s.n_act + blockIdx.x * blockDim.x + threadIdx.x; t < s.n; t += gridDim.x * blockDim.x) {
            const int i = s.act_order[t];
            if (p.typed)
                for (int u = 0; u < nbm; ++u) s.nseg[(size_t)i * BOUNCE_MAXT + u] = 0;
            s.nlong[i] = 0;
            s.nshort[i] = 0;
            s.refx[i] = s.qx[cur][i];
            s.refy[i] = s.qy[cur][i];
            s.refz[i] = s.qz[cur][i];
        }
    for (int t = t0 + blockIdx.x * wpb + warp; t < t1; t += gridDim.x * wpb) {
        const int i = split ? s.act_order[t] : t;
        const float4 hi = s.phi[cur][i];
        const int mi = s.mol[i];
        const int pm = filt ? p.jpart[s.type[i]] : -1;  // partner types of the row (all without the filter)
        int nr_tot;
        const int total_c = candidate_runs(s, p, hi, rb, rl, rp, nr_tot);
        __syncwarp();
        // window A: ww words centred on the atom's word, inside [0, nwords)
        const int wa = max(0, min((i >> 5) - ww / 2, nwords - ww));
        const int wz = min(wa + ww, nwords);
        int below[BOUNCE_MAXT], above[BOUNCE_MAXT];
#pragma unroll
        for (int t = 0; t < BOUNCE_MAXT; ++t) below[t] = above[t] = 0;
        int wmin = nwords, wmax = -1;  // words of the members outside the window
        int ulo = ww, uhi = -1;        // window words the members touched
        int lo_r = 0;  // run of candidate t: rp[lo_r] <= t < rp[lo_r + 1]; t only grows
        for (int t = lane; t < total_c; t += 32) {
            while (lo_r + 1 < nr_tot && rp[lo_r + 1] <= t) ++lo_r;
            const int idx = rb[lo_r] + (t - rp[lo_r]);
            const int j = s.cell_atoms[idx];
            if (j == i || s.cell_mol[idx] == mi || !((pm >> s.cell_type[idx]) & 1)) continue;
            float r2;
            if (!row_member(s, p, cur, i, hi, s.cell_phi[idx], j, r2)) continue;
            const int ty = p.typed ? s.cell_type[idx] : 0, w = j >> 5;
            if (w < wa) {
                wmin = min(wmin, w);
#pragma unroll
                for (int u = 0; u < BOUNCE_MAXT; ++u) below[u] += u == ty;
            } else if (w >= wz) {
                wmax = max(wmax, w);
#pragma unroll
                for (int u = 0; u < BOUNCE_MAXT; ++u) above[u] += u == ty;
            } else {
                atomicOr(&bm[(size_t)ty * ww + (w - wa)], 1u << (j & 31));
                ulo = min(ulo, w - wa);
                uhi = max(uhi, w - wa);
                // short rows: r < r_off + skin (rshort2 carries a 1e-4 margin)
                if (has_short && r2 < p.rshort2) atomicOr(&bs[w - wa], 1u << (j & 31));
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            wmin = min(wmin, __shfl_xor_sync(0xffffffffu, wmin, o));
            wmax = max(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
            ulo = min(ulo, __shfl_xor_sync(0xffffffffu, ulo, o));
            uhi = max(uhi, __shfl_xor_sync(0xffffffffu, uhi, o));
        }
        const bool outside = __any_sync(0xffffffffu, wmax >= 0 || wmin < nwords);
        if (outside) {
#pragma unroll
            for (int u = 0; u < BOUNCE_MAXT; ++u) {
                below[u] = warp_sum_i(below[u]);
                above[u] = warp_sum_i(above[u]);
            }
        }
        __syncwarp();
        // members of window A per type: popcounts over the touched words
        const int nu = uhi >= ulo ? uhi - ulo + 1 : 0;
        int inside[BOUNCE_MAXT], seg[BOUNCE_MAXT], total = 0;
#pragma unroll
        for (int u = 0; u < BOUNCE_MAXT; ++u) {
            int c = 0;
            if (u < nbm)
                for (int w = lane; w < nu; w += 32) c += __popc(bm[(size_t)u * ww + ulo + w]);
            inside[u] = warp_sum_i(c);
            seg[u] = total;
            total += u < nbm ? below[u] + inside[u] + above[u] : 0;
        }
        // window A in place (touched words only, cleared after): type group u
        // starts at seg[u], its members below the window first
        int* row = s.rows + (size_t)i * s.cap;
        for (int u = 0; u < nbm; ++u) {
            int off = 0;
#pragma unroll
            for (int v = 0; v < BOUNCE_MAXT; ++v) off = v == u ? seg[v] + below[v] : off;
            expand_bitmap(bm + (size_t)u * ww + ulo, nu, row + off, s.cap - off, wa + ulo);
        }
        const int ns = has_short ? expand_bitmap(bs + ulo, nu, s.srows + (size_t)i * s.caps, s.caps, wa + ulo) : 0;
        __syncwarp();
        for (int u = 0; u < nb; ++u)
            for (int w = lane; w < nu; w += 32) bm[(size_t)u * ww + ulo + w] = 0u;
        __syncwarp();
        // further windows: below window A (ascending from the lowest member), then above it
        if (outside)
            for (int side = 0; side < 2; ++side) {
                int w0 = side == 0 ? wmin : wz;
                const int wend = side == 0 ? wa : wmax + 1;
                int off[BOUNCE_MAXT];
#pragma unroll
                for (int u = 0; u < BOUNCE_MAXT; ++u) off[u] = seg[u] + (side == 0 ? 0 : below[u] + inside[u]);
                for (; w0 < wend; w0 += ww) {
                    const int w1 = min(w0 + ww, wend);
                    lo_r = 0;
                    for (int t = lane; t < total_c; t += 32) {
                        while (lo_r + 1 < nr_tot && rp[lo_r + 1] <= t) ++lo_r;
                        const int idx = rb[lo_r] + (t - rp[lo_r]);
                        const int j = s.cell_atoms[idx];
                        const int w = j >> 5;
                        if (w < w0 || w >= w1 || j == i || s.cell_mol[idx] == mi || !((pm >> s.cell_type[idx]) & 1))
                            continue;
                        float r2;
                        if (!row_member(s, p, cur, i, hi, s.cell_phi[idx], j, r2)) continue;
                        const int ty = p.typed ? s.cell_type[idx] : 0;
                        atomicOr(&bm[(size_t)ty * ww + (w - w0)], 1u << (j & 31));
                    }
                    __syncwarp();
                    for (int u = 0; u < nbm; ++u) {
                        int o = 0;
#pragma unroll
                        for (int v = 0; v < BOUNCE_MAXT; ++v) o = v == u ? off[v] : o;
                        const int c = expand_bitmap(bm + (size_t)u * ww, w1 - w0, row + o, s.cap - o, w0);
#pragma unroll
                        for (int v = 0; v < BOUNCE_MAXT; ++v) off[v] += v == u ? c : 0;
                    }
                    __syncwarp();
                    for (int w = lane; w < nbm * ww; w += 32) bm[w] = 0u;
                    __syncwarp();
                }
            }
        if (lane == 0) {
            if (p.typed)
                for (int u = 0; u < nbm; ++u) {
                    int c = 0;
#pragma unroll
                    for (int v = 0; v < BOUNCE_MAXT; ++v) c = v == u ? below[v] + inside[v] + above[v] : c;
                    s.nseg[(size_t)i * BOUNCE_MAXT + u] = c;
                }
            s.nlong[i] = min(total, s.cap);
            if (total > s.cap) atomicOr(s.err, BERR_LIST_OVERFLOW);
            s.nshort[i] = min(ns, s.caps);
            if (ns > s.caps) atomicOr(s.err, BERR_SHORT_OVERFLOW);
            if (own) {
                s.refx[i] = s.qx[cur][i];
                s.refy[i] = s.qy[cur][i];
                s.refz[i] = s.qz[cur][i];
            }
        }
        __syncwarp();
    }
    if (last_cta(&s.done_ctr[1]) && own) *s.rebuild = 0;
}

// Rows of a batch of independent all-pairs replicas: every atom of the same
// replica outside the own molecule, ascending (no distance test: replicas
// have no cutoff), then the short rows and reference positions as above.
__global__ void k_rows_batch(DevSys s, Params p, int step_off, int force, int mode_in) {
    if (!pending(s, force)) return;
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    const int cur = (int)((*s.step_base + step_off) & 1);
    const bool filt = (mode_in & ROWS_FILTER) != 0;
    const bool own = (mode_in & 7) != ROWS_IDLE && (mode_in & 7) != ROWS_READER;
    if (blockIdx.x == 0 && threadIdx.x == 0 && own) atomicAdd(&s.cnt[CNT_REBUILDS], 1ull);
    for (int i = blockIdx.x * wpb + (threadIdx.x >> 5); i < s.n; i += gridDim.x * wpb) {
        const int r = s.rep_of[i], b = s.rep_off[r], e = s.rep_off[r + 1], mi = s.mol[i];
        const int pm = filt ? p.jpart[s.type[i]] : -1;  // partner types of the row (all without the filter)
        int* row = s.rows + (size_t)i * s.cap;
        int total = 0;
        const int ngroups = p.typed ? p.n_types : 1;
        for (int tb = 0; tb < ngroups; ++tb) {  // typed rows: one pass per partner type
            const int before = total;
            for (int j0 = b; j0 < e; j0 += 32) {
                const int j = j0 + lane;
                const bool keep = j < e && s.mol[j] != mi && (!p.typed || s.type[j] == tb) && ((pm >> s.type[j]) & 1);
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
            if (own) {
                s.refx[i] = s.qx[cur][i];
                s.refy[i] = s.qy[cur][i];
                s.refz[i] = s.qz[cur][i];
            }
        }
        __syncwarp();
    }
    if (last_cta(&s.done_ctr[1]) && own) *s.rebuild = 0;
}

__global__ void k_flag_moved(DevSys s, Params p, int cur) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < s.n; i += gridDim.x * blockDim.x) {
        const double ex = s.qx[cur][i] - s.refx[i], ey = s.qy[cur][i] - s.refy[i], ez = s.qz[cur][i] - s.refz[i];
        if (((s.rows_move >> s.type[i]) & 1) && ex * ex + ey * ey + ez * ez > p.skin_half2) atomicOr(s.rebuild, 1);
    }
}

}  // namespace

void launch_flag_moved(const DevSys& s, const Params& p, int cur, cudaStream_t st) {
    k_flag_moved<<<(s.n + 255) / 256, 256, 0, st>>>(s, p, cur);
}

void launch_rebuild(const DevSys& s, const Params& p, int step_off, bool force, int window_words, size_t bitmap_bytes,
                    int mode, cudaStream_t st) {
    const int f = force ? 1 : 0;
    if (s.rep_of) {
        const int wpb = 8;
        launch_chained(k_rows_batch, (s.n + wpb - 1) / wpb, wpb * 32, 0, st, s, p, step_off, f, mode);
        return;
    }
    const int tb = 1024;
    const int gb = (s.n + tb - 1) / tb;
    launch_chained(k_cells_count, gb, tb, 0, st, s, p, step_off, f, mode);
    launch_chained(k_cells_scatter, gb, tb, 0, st, s, p, step_off, f, mode);
    // warp per atom, 8 warps per CTA, a grid-stride loop over one wave of CTAs
    const int per_sm = std::max(1, std::min(8, (int)((227u << 10) / std::max<size_t>(bitmap_bytes, 1))));
    const int blocks = std::min((s.n + 7) / 8, 152 * per_sm);
    launch_chained(k_rows_warp, blocks, 256, bitmap_bytes, st, s, p, step_off, f, window_words, mode);
}

void nlist_set_smem_limit(size_t bytes) {
    cudaFuncSetAttribute(k_rows_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}
