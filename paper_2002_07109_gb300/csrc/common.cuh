// Shared device-side definitions of the BOUNCE library: the system view
// passed to every kernel, the Philox4x32-10 generator, the FP32 exp(-x) and
// Poisson inversion used by the jump step, and the FP32 pair terms.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#define BOUNCE_MAXT 4
#define BOUNCE_GROUP 32                // atoms per CTA in the fused step kernels
#define BOUNCE_POISSON_SLOT 0x80000000u
#define BOUNCE_STREAM_O 0u
#define BOUNCE_STREAM_J1 1u
#define BOUNCE_STREAM_J2 2u

// Error bits set by kernels (ctx->err).
#define BERR_LIST_OVERFLOW 1
#define BERR_SHORT_OVERFLOW 2
#define BERR_RATE 4               // a jump proposal mean was not finite or above 1e6

// Counter slots (unsigned long long).
enum { CNT_PROPOSALS = 0, CNT_ACCEPTS, CNT_NEAR, CNT_REBUILDS, CNT_SHORT_PAIRS, CNT_FULL_PAIRS, CNT_N };

constexpr double KCOUL_D = 332.063713;
constexpr double KB_D = 0.0019872041;
constexpr double ACCEL_D = 4.184e-4;

// Cluster-pair structure of the pair sums (finite cutoff, one system):
// atoms binned into columns of a grid over (x, y), sorted by z inside each
// column and cut into clusters of BOUNCE_CL consecutive atoms; cluster I of
// column col has id col * maxcl + k and owns slots id * BOUNCE_CL + t.  The
// list of cluster I holds every atom of a cluster J >= I that lies within a
// search radius (r_c, or the short-range radius, plus the skin) of I's
// bounding box, with the periodic image code of the pair; the pair kernel
// sums both sides of every pair once (Newton's third law) into int64
// fixed-point accumulators, one per slot and component.
#define BOUNCE_CL 8
#ifndef BOUNCE_CL_EPW
#define BOUNCE_CL_EPW 512          // list entries per work item of the pair kernel (one item per
                                   // cluster on the water box: fewer i-side reductions)
#endif
#define BOUNCE_CL_MAXCOL 1024      // atoms per column (one CTA sorts a column in shared memory)
constexpr double CL_FIX = 4294967296.0;        // fixed-point scale 2^32 of the accumulators
constexpr double CL_UNFIX = 2.3283064365386963e-10;  // 2^-32

struct DevClu {
    int on;                  // the pair sums run over clusters
    int ncx, ncy, ncol;      // column grid
    float ox, oy;            // grid origin (droplets)
    float ihx, ihy;          // inverse column edges
    int maxcl;               // cluster ids per column
    int maxcol;              // atoms per column (<= BOUNCE_CL_MAXCOL)
    int nlists;              // 1, or 2 with a distinct short-range list
    int capj[2];             // entries per cluster of each list
    float rs2[2];            // squared search radii of the lists (with margins)
    float rsx[2];            // the radii themselves
    double cskin_half2;      // rebuild when an atom moved more than skin/2 since the build
    int* col_count;          // [ncol]
    int* col_start;          // [ncol + 1]
    int* col_fill;           // [ncol]
    int* col_atoms;          // [n] atoms in column order
    int* col_ncl;            // [ncol] clusters of each column
    int* atom_col;           // [n] column of each atom at the build
    int* cl_atom;            // [ncl * CL] atom of each slot (-1: padding)
    int* a2s;                // [n] slot of each atom
    float4* sphi[2];         // slot-ordered copies of phi / plo (same buffers as the positions)
    float4* splo[2];
    int* smol;               // [ncl * CL] molecule id (-1: padding)
    float4* bb_lo;           // [ncl] bounding box of each cluster (high FP32 parts)
    float4* bb_hi;
    int* lst[2];             // [ncl * capj] slot of j | image code << 27
    int* lcnt[2];            // [ncl] entries of each cluster
    unsigned long long* acc; // [3 * ncl * CL] fixed-point gradient sums (x, y, z blocks)
    double* crefx;           // [n] positions at the build
    double* crefy;
    double* crefz;
    double* cofx;            // [n] periodic image offset L floor(q / L) of each atom at the build:
    double* cofy;            //     the slot copies keep q - cof until the next build, so that the
    double* cofz;            //     image codes of the lists stay valid when atoms cross a face
    int* rebuild;            // 1 = the clusters must be rebuilt before the next pair sums
    unsigned int* done_ctr;  // [4] finished-CTA counters (zero between launches)
    // pruned lists: the entries of lst within r + prune skin of some atom of
    // I at the last prune, valid while no atom moved half the prune skin
    int* plst[2];            // [ncl * capj] same layout as lst
    int* pcnt[2];            // [ncl]
    int2* pitems[2];         // (I, first entry) of each work item of the pruned lists, in allocation order
    int* pnitems;            // [2] work items, [2..3] their allocation counters, [4..5] the
                             //     pair kernel's fetch counters (zero between launches)
    int capitems;            // work items per list
    float4* pref;            // [ncl * CL] slot positions (high parts) at the last prune
    float prs2[2];           // squared prune radii (r_c or r'' plus the prune skin, with a margin)
    float pdisp2;            // squared displacement that triggers the next prune
    int* prune;              // 1 = prune before the next pair sums
};

// All-pairs sums (systems without a cutoff): static items (first i, count,
// first j, count) of 32-atom i-tiles against j-blocks of one replica, and
// atom-indexed int64 fixed-point accumulators.
struct DevTile {
    int on;                  // the pair sums over all pairs run over tiles
    int nitems;
    int blocks;              // resident grid of the tile kernel
    int tj;                  // atoms per j-block
    const int4* items;
    unsigned long long* acc; // [3 n] (x, y, z blocks)
};

// Device pointers of one system (passed by value).
struct DevSys {
    int n;
    double* qx[2];
    double* qy[2];
    double* qz[2];
    float4* phi[2];  // (x, y, z) high FP32 part of the (wrapped) position, w = charge
    float4* plo[2];  // (x, y, z) low FP32 part, w = type (bit pattern of an int)
    double* vx;
    double* vy;
    double* vz;
    const double* kick;  // 4.184e-4 / m
    const double* osd;   // sqrt((1 - c1^2) k_B T 4.184e-4 / m)
    const int* type;
    const int* mol;
    // bonded terms touching each atom: bt_off[n + 1], bt_idx (role, o1, o2, -), bt_par (k, x0)
    const int* bt_off;
    const int4* bt_idx;
    const float2* bt_par;
    // candidate rows (r < r_list) and short rows (r < r_off + skin)
    int* nlong;
    int* rows;
    int cap;
    int* nseg;      // [n][BOUNCE_MAXT] candidates of each type in the row (typed rows)
    int* nshort;
    int* srows;
    int caps;
    double* refx;
    double* refy;
    double* refz;
    // cell grid
    int* cell_count;
    int* cell_start;
    int* cell_fill;
    int* cell_atoms;
    float4* cell_phi;  // high position parts in cell order (coalesced candidate reads)
    float4* g0;        // pair-sum gradient of each atom from k_pairs (x, y, z; w = row entries, int bits)
    unsigned int* done_ctr;  // [2] finished-CTA counters of the rebuild kernels (zero between launches)
    int* cell_mol;     // molecule ids in cell order
    int* cell_type;    // atom types in cell order
    int ncx, ncy, ncz;
    float ox, oy, oz;        // grid origin (droplets)
    float ihx, ihy, ihz;     // inverse cell edges
    float hx, hy, hz;        // cell edges
    int mx, my, mz;          // search reach in cells (ceil(r_list / edge))
    // flags and counters
    int* rebuild;            // 1 = rows must be rebuilt before the next evaluation
    int* err;
    unsigned long long* cnt;
    const long long* step_base;
    const double* grecip;    // reciprocal + exclusion gradient [3 n] (SoA), null without PME
    // batched independent replicas (null for one system): replica of each
    // atom, its index inside the replica and each replica's Philox key
    const int* rep_of;
    const int* local_idx;
    const uint2* rep_key;
    const int* rep_off;      // [replicas + 1] first atom of each replica
    DevClu cl;               // cluster-pair structure (cl.on = 0: pair sums over the rows)
    DevTile tl;              // all-pairs tiles (systems without a cutoff)
    const int* act_order;    // [n] atoms whose type has L* > 0 (ascending), then the others
    int n_act;               // atoms that can propose
    int rows_flag;           // the step kernel raises `rebuild` for the rows (0 in BAOAB runs on clusters)
    unsigned rows_move;      // types whose displacement raises `rebuild` (all of them unless the
                             //     jump rows keep only the partners a jump can draw)
    int lite;                // thread-per-atom step kernel (rare jump proposals)
};

// Smooth particle-mesh Ewald state (periodic boxes with a reciprocal part).
struct DevPme {
    int K[3];
    int order;
    double L[3];
    double iL[3], KL[3];         // 1 / L and K / L per axis (no FP64 division per atom)
    float beta, two_b_sqrtpi;
    unsigned long long* qgrid;   // int64 fixed-point charge grid (2^40 scale)
    float2* cgrid;               // complex work grid
    const float* bc;             // influence function B(m) C(m)
    double* grad;                // [3 n] SoA gradient of E_recip + E_excl
    double* eexcl;               // [n] exclusion energy per atom (pairs j > i)
    double* eterm;               // [256] energy partials of the convolution
    const int* ex_off;           // [n + 1] same-molecule partners of each atom
    const int* ex_idx;
};

// Scalar parameters (passed by value; fits the kernel parameter space).
struct Params {
    float c12[BOUNCE_MAXT * BOUNCE_MAXT];  // 4 eps sigma^12
    float c6[BOUNCE_MAXT * BOUNCE_MAXT];   // 4 eps sigma^6
    float kcoul;
    float rc2_lo, rc2_hi;  // FP32 screening band around r_c^2 (+inf = no cutoff)
    double rc2_d;          // exact FP64 cutoff test r^2 < r_c^2
    float r_on, inv_span;
    int chi_step;        // 1: chi = indicator of [r_off, inf)
    float r_off;
    float ebeta, e2b_sqrtpi;  // Ewald beta and 2 beta / sqrt(pi); ebeta = 0: bare Coulomb
    int periodic;
    float Lhi[3], Llo[3], invL[3];
    double Ld[3], iLd[3];        // box edges and their inverses (FP64)
    float rlist2_lo, rlist2_hi;  // FP32 screening band around r_list^2
    double rlist2_d;             // exact FP64 threshold r_list^2 (+inf = all)
    float rshort2;               // short-row threshold
    float rcull;                 // r_list with a safety margin for cell culling (+inf = all)
    int coul_jump;               // 1: Coulomb is switched by chi like LJ; 0: Coulomb wholly in F_0
    int typed;                   // per-type-pair bounds with the two-stage partner choice
    int jpart[BOUNCE_MAXT];      // jump rows (ROWS_FILTER): types an atom of type a can draw, as a bitmask
    int jcells;                  // jump rows: types placed in the cells (every type some row can hold)
    int n_types;
    uint32_t lq[BOUNCE_MAXT * BOUNCE_MAXT];  // integer weights Lq_ab of the partner types
    uint32_t lq_m[BOUNCE_MAXT * BOUNCE_MAXT];  // x / Lq_ab = (t + ((x - t) >> 1)) >> lq_s, t = umulhi(lq_m, x)
    uint32_t lq_s[BOUNCE_MAXT * BOUNCE_MAXT];  //   (Granlund-Montgomery division by an invariant integer)
    double lt_d[BOUNCE_MAXT * BOUNCE_MAXT];  // their bounds Lt_ab = Lq_ab L*_a 2^-16
    float Lstar_f[BOUNCE_MAXT];
    double Lstar_d[BOUNCE_MAXT];
    double beta;
    double dt;
    float beta_f, dt_half_f;     // beta and dt / 2 in FP32 (the jump step's bound of the Poisson mean)
    double c1;
    double skin_half2;
    uint32_t key0, key1;
};

// ------------------------------------------------------------------ Philox
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of two
// 32x32->64 multiplies with the round constants, key bumped by the Weyl
// constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// Counter (slot, atom, step mod 2^32, stream << 24 | step >> 32 mod 2^24).
__device__ __forceinline__ uint4 rng_draw(const Params& p, uint32_t slot, uint32_t atom, long long step,
                                          uint32_t stream) {
    uint4 c = make_uint4(slot, atom, (uint32_t)(step & 0xFFFFFFFFll),
                         (stream << 24) | (uint32_t)((step >> 32) & 0xFFFFFFll));
    return philox4x32_10(c, p.key0, p.key1);
}

// Draw for atom i: its replica's key and its index inside the replica when
// the context holds a batch, the run key and the global index otherwise.
__device__ __forceinline__ uint4 rng_atom(const DevSys& s, const Params& p, uint32_t slot, int i, long long step,
                                          uint32_t stream) {
    uint4 c = make_uint4(slot, 0u, (uint32_t)(step & 0xFFFFFFFFll), (stream << 24) | (uint32_t)((step >> 32) & 0xFFFFFFll));
    if (s.rep_of) {
        const uint2 k = s.rep_key[s.rep_of[i]];
        c.y = (uint32_t)s.local_idx[i];
        return philox4x32_10(c, k.x, k.y);
    }
    c.y = (uint32_t)i;
    return philox4x32_10(c, p.key0, p.key1);
}

__device__ __forceinline__ float u24(uint32_t x) { return (float)(x >> 8) * 5.9604644775390625e-08f; }
__device__ __forceinline__ float u24_open0(uint32_t x) { return (float)((x >> 8) + 1u) * 5.9604644775390625e-08f; }
__device__ __forceinline__ double u53(uint32_t x1, uint32_t x2) {
    return __dmul_rn(__dadd_rn(__dmul_rn((double)(x1 >> 5), 67108864.0), (double)(x2 >> 6)),
                     1.1102230246251565e-16);
}

// ------------------------------------------------------- FP32 exp(-x), Poisson
// exp(-x) for x in [0, 32]: x = n ln2 + r with n = floor(x log2 e + 1/2)
// (two-constant reduction), exp(-r) by its Taylor polynomial of degree 7
// (coefficients (-1)^k / k!), scaled by 2^-n.  Every operation is an explicit
// round-to-nearest FP32 operation so the result does not depend on
// contraction choices.
__device__ __forceinline__ float expneg_f32(float x) {
    const float LOG2E = (float)(1.0 / 0.6931471805599453094);
    const float LN2_HI = 0.693145751953125f;
    const float LN2_LO = (float)(0.6931471805599453094 - 0.693145751953125);
    const float C0 = 1.0f, C1 = -1.0f, C2 = (float)(1.0 / 2.0), C3 = (float)(-1.0 / 6.0),
                C4 = (float)(1.0 / 24.0), C5 = (float)(-1.0 / 120.0), C6 = (float)(1.0 / 720.0),
                C7 = (float)(-1.0 / 5040.0);
    float t = __fmul_rn(x, LOG2E);
    float n = floorf(__fadd_rn(t, 0.5f));
    float r = __fsub_rn(__fsub_rn(x, __fmul_rn(n, LN2_HI)), __fmul_rn(n, LN2_LO));
    float q = C7;
    q = __fadd_rn(__fmul_rn(q, r), C6);
    q = __fadd_rn(__fmul_rn(q, r), C5);
    q = __fadd_rn(__fmul_rn(q, r), C4);
    q = __fadd_rn(__fmul_rn(q, r), C3);
    q = __fadd_rn(__fmul_rn(q, r), C2);
    q = __fadd_rn(__fmul_rn(q, r), C1);
    q = __fadd_rn(__fmul_rn(q, r), C0);
    return __fmul_rn(q, ldexpf(1.0f, -(int)n));
}

// One Poisson(mu_c) count by sequential search of the CDF in FP32
// (mu_c <= 16); stops when the CDF passes u, when adding a term no longer
// changes it, or at k = 128.
__device__ __forceinline__ int poisson_invert_f32(float u, float mu_c) {
    float p = expneg_f32(mu_c);
    float cdf = p;
    int k = 0;
    while (u > cdf && k < 128) {
        ++k;
        float pk = __fmul_rn(__fmul_rn(p, mu_c), __frcp_rn((float)k));
        float cn = __fadd_rn(cdf, pk);
        if (cn == cdf) break;
        p = pk;
        cdf = cn;
    }
    return k;
}

// x wrapped into [0, L): the multiple of L from the product with 1/L (no
// FP64 division on the per-step path), moved by one where the product's
// rounding put x on the wrong side of a multiple.
__device__ __forceinline__ double wrap_box(double x, double L, double iL) {
    double w = x - L * floor(x * iL);
    if (w < 0.0) w += L;
    else if (w >= L) w -= L;
    return w;
}

// ------------------------------------------------------------- pair terms
// Displacement q_i - q_j from the split FP32 positions (hi + lo), minimum
// image under periodic boundaries.
__device__ __forceinline__ float3 pair_disp(const Params& p, float4 hi, float4 lo, float4 hj, float4 lj) {
    float dx = hi.x - hj.x, dy = hi.y - hj.y, dz = hi.z - hj.z;
    float ex = lo.x - lj.x, ey = lo.y - lj.y, ez = lo.z - lj.z;
    if (p.periodic) {
        float kx = rintf(dx * p.invL[0]), ky = rintf(dy * p.invL[1]), kz = rintf(dz * p.invL[2]);
        dx = fmaf(-kx, p.Lhi[0], dx);
        dy = fmaf(-ky, p.Lhi[1], dy);
        dz = fmaf(-kz, p.Lhi[2], dz);
        ex = fmaf(-kx, p.Llo[0], ex);
        ey = fmaf(-ky, p.Llo[1], ey);
        ez = fmaf(-kz, p.Llo[2], ez);
    }
    return make_float3(dx + ex, dy + ey, dz + ez);
}

// 1/sqrt(r2) to about 1 ulp: the hardware estimate refined by one Newton step.
__device__ __forceinline__ float rsqrt_nr(float r2) {
    const float y = rsqrtf(r2);
    return y * fmaf(-0.5f * r2 * y, y, 1.5f);
}

// Coulomb (or Ewald direct) part wc and LJ part wl of W'(r) / r of one pair,
// r2 < rc2 assumed; r = r2 / sqrt(r2) from the same reciprocal square root.
__device__ __forceinline__ void pair_dW_parts(const Params& p, float r2, float qq, int tp, float& wc, float& wl,
                                              float& r) {
    float ir = rsqrt_nr(r2);
    float ir2 = ir * ir;
    r = r2 * ir;
    if (p.ebeta > 0.f) {
        float br = p.ebeta * r;
        wc = -qq * (erfcf(br) * ir2 + p.e2b_sqrtpi * __expf(-br * br) * ir) * ir;
    } else {
        wc = -qq * ir2 * ir;
    }
    wl = 0.f;
    float c12 = p.c12[tp];
    if (c12 != 0.f) {
        float ir6 = ir2 * ir2 * ir2;
        wl = -((12.f * c12 * ir6 - 6.f * p.c6[tp]) * ir6 * ir2);
    }
}

// W'(r) / r of one pair (Coulomb or Ewald direct + LJ), r2 < rc2 assumed.
__device__ __forceinline__ float pair_dW_over_r(const Params& p, float r2, float qq, int tp) {
    float wc, wl, r;
    pair_dW_parts(p, r2, qq, tp, wc, wl, r);
    return wc + wl;
}

// W'/r split into the part switched by chi (sw) and the part that always
// stays in F_0 (fixed): (all, 0), or (LJ, Coulomb) when Coulomb is kept out
// of the jumps.  One evaluation of the pair terms either way; r as above.
__device__ __forceinline__ void pair_dW_split(const Params& p, float r2, float qq, int tp, float& sw, float& fixed,
                                              float& r) {
    float wc, wl;
    pair_dW_parts(p, r2, qq, tp, wc, wl, r);
    if (p.coul_jump) {
        sw = wc + wl;
        fixed = 0.f;
    } else {
        sw = wl;
        fixed = wc;
    }
}

// Switching function chi(r) (quintic smoothstep on [r', r'']).
__device__ __forceinline__ float chi_of(const Params& p, float r);

// W'/r of the F_0 share of one pair: (1 - chi) times the switched part plus
// the fixed part (pair_dW_split).  The switched part, LJ included, is not
// evaluated at or beyond r'', where 1 - chi = 0; the result equals
// sw (1 - chi) + fixed there too.
__device__ __forceinline__ float pair_dW_f0(const Params& p, float r2, float qq, int tp) {
    const float ir = rsqrt_nr(r2);
    const float ir2 = ir * ir;
    const float r = r2 * ir;
    float wc;
    if (p.ebeta > 0.f) {
        const float br = p.ebeta * r;
        wc = -qq * (erfcf(br) * ir2 + p.e2b_sqrtpi * __expf(-br * br) * ir) * ir;
    } else {
        wc = -qq * ir2 * ir;
    }
    const float fixed = p.coul_jump ? 0.f : wc;
    if (!(r < p.r_off)) return fixed;
    float wl = 0.f;
    const float c12 = p.c12[tp];
    if (c12 != 0.f) {
        const float ir6 = ir2 * ir2 * ir2;
        wl = -((12.f * c12 * ir6 - 6.f * p.c6[tp]) * ir6 * ir2);
    }
    const float sw = p.coul_jump ? wc + wl : wl;
    return sw * (1.f - chi_of(p, r)) + fixed;
}

// Switching function chi(r) (quintic smoothstep on [r', r''])
__device__ __forceinline__ float chi_of(const Params& p, float r) {
    if (p.chi_step) return r >= p.r_off ? 1.f : 0.f;
    float s = fminf(fmaxf((r - p.r_on) * p.inv_span, 0.f), 1.f);
    return s * s * s * (10.f + s * (-15.f + 6.f * s));
}

// 1: the pair sums take erfc from the CUDA library instead of 7.1.26
#ifndef CL_LIBRARY_ERFC
#define CL_LIBRARY_ERFC 0
#endif

// erfc(x) e^{x^2} for x >= 0 by Abramowitz and Stegun, Handbook of
// Mathematical Functions, 7.1.26: t = 1/(1 + p x), t (a1 + t (a2 + t (a3 +
// t (a4 + t a5)))); absolute error of erfc(x) below 1.5e-7.  The pair sums
// use it (with the exp(-x^2) they need for the derivative anyway); the jump
// step keeps the library erfcf.
__device__ __forceinline__ float erfc_scaled_as(float x) {
    const float t = __fdividef(1.f, fmaf(0.3275911f, x, 1.f));
    return t * fmaf(t, fmaf(t, fmaf(t, fmaf(t, 1.061405429f, -1.453152027f), 1.421413741f), -0.284496736f),
                    0.254829592f);
}

// W'(r)/r of one pair for the pair sums (cluster and tile kernels), without
// branches on the pair's own values (every lane of a warp runs it; masked
// pairs pass r2 = 1):
// PART 5 the full W', PART 3 the F_0 share (1 - chi) W'_sw + W'_fixed.
template <int PART>
__device__ __forceinline__ float pairsum_w(const Params& p, float r2, float qq, float c12, float c6) {
    const float ir = rsqrt_nr(r2);
    const float ir2 = ir * ir;
    const float r = r2 * ir;
    float wc;
    if (p.ebeta > 0.f) {
        const float x = p.ebeta * r;
        const float e = __expf(-x * x);
#if CL_LIBRARY_ERFC
        wc = -qq * (erfcf(x) * ir2 + p.e2b_sqrtpi * e * ir) * ir;
#else
        wc = -qq * (erfc_scaled_as(x) * e * ir2 + p.e2b_sqrtpi * e * ir) * ir;
#endif
    } else {
        wc = -qq * ir2 * ir;
    }
    const float ir6 = ir2 * ir2 * ir2;
    const float wl = -((12.f * c12 * ir6 - 6.f * c6) * ir6 * ir2);
    // explicit roundings: the F_0 share with chi = 0 equals the full term bit
    // for bit whatever the compiler contracts around it
    const float wsum = __fadd_rn(wc, wl);
    if (PART == 5) return wsum;
    float chi;
    if (p.chi_step) {
        chi = r >= p.r_off ? 1.f : 0.f;
    } else {
        const float sx = fminf(fmaxf((r - p.r_on) * p.inv_span, 0.f), 1.f);
        chi = sx * sx * sx * fmaf(sx, fmaf(6.f, sx, -15.f), 10.f);
    }
    return p.coul_jump ? __fmul_rn(wsum, 1.f - chi) : __fadd_rn(__fmul_rn(wl, 1.f - chi), wc);
}

// Pair energy W(r) components (Coulomb or erfc, LJ), r2 < rc2 assumed.
__device__ __forceinline__ void pair_W(const Params& p, float r2, float qq, int tp, float& ec, float& el) {
    float ir = rsqrt_nr(r2);
    if (p.ebeta > 0.f) {
        float r = r2 * ir;
        ec = qq * erfcf(p.ebeta * r) * ir;
    } else {
        ec = qq * ir;
    }
    float c12 = p.c12[tp];
    el = 0.f;
    if (c12 != 0.f) {
        float ir2 = ir * ir;
        float ir6 = ir2 * ir2 * ir2;
        el = (c12 * ir6 - p.c6[tp]) * ir6;
    }
}

// Exact FP64 r_ij^2 with the minimum image d - L rint(d / L), evaluated as
// (dx dx + dy dy) + dz dz with round-to-nearest and no contraction.
__device__ __forceinline__ double exact_r2(const DevSys& s, const Params& p, int cur, int i, int j) {
    double dx = __dsub_rn(s.qx[cur][i], s.qx[cur][j]);
    double dy = __dsub_rn(s.qy[cur][i], s.qy[cur][j]);
    double dz = __dsub_rn(s.qz[cur][i], s.qz[cur][j]);
    if (p.periodic) {
        dx = __dsub_rn(dx, __dmul_rn(p.Ld[0], rint(__ddiv_rn(dx, p.Ld[0]))));
        dy = __dsub_rn(dy, __dmul_rn(p.Ld[1], rint(__ddiv_rn(dy, p.Ld[1]))));
        dz = __dsub_rn(dz, __dmul_rn(p.Ld[2], rint(__ddiv_rn(dz, p.Ld[2]))));
    }
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// Pair cutoff test r^2 < r_c^2: decided in FP32 outside a narrow band around
// r_c^2 and exactly in FP64 inside it.
__device__ __forceinline__ bool inside_cut(const DevSys& s, const Params& p, int cur, int i, int j, float r2f) {
    if (r2f < p.rc2_lo) return true;
    if (!(r2f <= p.rc2_hi)) return false;
    return exact_r2(s, p, cur, i, j) < p.rc2_d;
}

__device__ __forceinline__ int type_of(float4 lo) { return __float_as_int(lo.w); }

// round(v 2^S) as a two's-complement 64-bit integer for the fixed-point
// accumulators: the FP32 product with 2^S is exact, the conversion rounds to
// nearest (ties to even); |v| is clamped to 2^(63 - S), where the conversion
// would saturate.  Integer sums of these do not depend on the order of the
// additions.
template <int S>
__device__ __forceinline__ unsigned long long fix_round(float v) {
    constexpr float scale = (float)(1ull << S);
    constexpr float vmax = (float)(1ull << (63 - S));
    return (unsigned long long)__float2ll_rn(fminf(fmaxf(v, -vmax), vmax) * scale);
}

__device__ __forceinline__ float warp_sum_f(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}
__device__ __forceinline__ int warp_sum_i(int x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Gradient on atom i of the bonded terms listed for it (FP32 from split
// positions).  role 0: bond to o1; role 1: angle end (vertex o1, other end
// o2); role 2: angle vertex (ends o1, o2).
__device__ __forceinline__ float3 bonded_grad(const Params& p, const DevSys& s, int cur, int i, int4 t, float2 kp) {
    float4 hi = s.phi[cur][i], lo = s.plo[cur][i];
    float3 g = make_float3(0.f, 0.f, 0.f);
    if (t.x == 0) {
        float3 d = pair_disp(p, hi, lo, s.phi[cur][t.y], s.plo[cur][t.y]);
        float r = sqrtf(d.x * d.x + d.y * d.y + d.z * d.z);
        float c = 2.f * kp.x * (r - kp.y) / r;
        g = make_float3(c * d.x, c * d.y, c * d.z);
    } else {
        // angle a-b-c with b the vertex
        int a, b, c;
        if (t.x == 1) { a = i; b = t.y; c = t.z; } else { a = t.y; b = i; c = t.z; }
        float4 hb = s.phi[cur][b], lb = s.plo[cur][b];
        float3 u = pair_disp(p, s.phi[cur][a], s.plo[cur][a], hb, lb);
        float3 w = pair_disp(p, s.phi[cur][c], s.plo[cur][c], hb, lb);
        float nu2 = u.x * u.x + u.y * u.y + u.z * u.z, nw2 = w.x * w.x + w.y * w.y + w.z * w.z;
        float inuw = rsqrt_nr(nu2 * nw2);
        float cs = (u.x * w.x + u.y * w.y + u.z * w.z) * inuw;
        cs = fminf(fmaxf(cs, -1.f), 1.f);
        float th = acosf(cs);
        float sn = sqrtf(fmaxf(1.f - cs * cs, 1e-12f));
        float dE = 2.f * kp.x * (th - kp.y);
        // d theta / d a = -(w/(|u||w|) - cos u/|u|^2) / sin ; same for c with u <-> w
        float fa = -dE / sn;
        float3 ga = make_float3(fa * (w.x * inuw - cs * u.x / nu2), fa * (w.y * inuw - cs * u.y / nu2),
                                fa * (w.z * inuw - cs * u.z / nu2));
        if (t.x == 1) {
            g = ga;
        } else {
            float3 gc = make_float3(fa * (u.x * inuw - cs * w.x / nw2), fa * (u.y * inuw - cs * w.y / nw2),
                                    fa * (u.z * inuw - cs * w.z / nw2));
            g = make_float3(-(ga.x + gc.x), -(ga.y + gc.y), -(ga.z + gc.z));
        }
    }
    return g;
}

// Programmatic dependent launch of the per-step kernel chain (row-rebuild
// gates, step kernel, step counter): a kernel launched with launch_chained
// may be scheduled while its predecessor in the stream still runs.  It waits
// here until the predecessor has completed and its writes are visible, before
// reading anything, and then lets its own successor be scheduled.  Without a
// programmatic predecessor the wait returns at once.
__device__ __forceinline__ void chain_enter() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_chained(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                  Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Row-build modes of launch_rebuild (see k_rows_warp); ROWS_FILTER may be
// added to ROWS_ALL or ROWS_ACTIVE: rows of the jump step that keep only the
// partners a jump can draw (Params::jpart).
constexpr int ROWS_ALL = 0, ROWS_ACTIVE = 1, ROWS_IDLE = 2, ROWS_READER = 3, ROWS_FILTER = 8;

// Launchers implemented in the .cu files.
void launch_rebuild(const DevSys& s, const Params& p, int step_off, bool force, int window_words, size_t bitmap_bytes,
                    int mode, cudaStream_t st);
void launch_step(const DevSys& s, const Params& p, int integrator, int variant, int step_off, double hr,
                 double hout, cudaStream_t st);
// launch_step in two parts (for per-kernel timing): the pair sums, then the step kernel.
int launch_step_pairs(const DevSys& s, const Params& p, int integrator, int step_off, double hout, cudaStream_t st);
void launch_step_kernel(const DevSys& s, const Params& p, int integrator, int variant, int step_off, double hr,
                        double hout, int pre, cudaStream_t st);
// energy: also the FP64 energy partials of the convolution (bounce_get_energies)
void launch_pme(const DevSys& s, const Params& p, const DevPme& m, int step_off, cudaStream_t st, bool energy = false);
void launch_pme_energy(const DevPme& m, int n, double* out, cudaStream_t st);
void launch_gradient(const DevSys& s, const Params& p, int part, int cur, double* out, cudaStream_t st);
void launch_jump_half(const DevSys& s, const Params& p, int cur, long long step, int stream_id, int* M, int* nacc,
                      cudaStream_t st);
void launch_energies(const DevSys& s, const Params& p, int cur, double* terms, cudaStream_t st);
void launch_advance_step(const DevSys& s, long long by, cudaStream_t st);
void launch_pack_positions(const DevSys& s, const Params& p, int cur, cudaStream_t st);
void launch_state_in(const DevSys& s, const double* q, const double* v, int cur, cudaStream_t st);
void launch_state_out(const DevSys& s, double* q, double* v, cudaStream_t st);
// Raises the rebuild flag when an atom at positions `cur` lies more than
// skin/2 from its position at the last row build (the step kernel's test).
void launch_flag_moved(const DevSys& s, const Params& p, int cur, cudaStream_t st);
// Cluster-pair path (cluster.cu): gated rebuild of the clusters and lists,
// the pair sums of `part` (3: F_0 share, 5: full pairs) over list `list`
// into the fixed-point accumulators, and their read-out (added to out[3n],
// accumulators cleared).
void launch_cluster_rebuild(const DevSys& s, const Params& p, int step_off, bool force, cudaStream_t st);
// sizes the pair kernel's resident grid once (outside any graph capture)
void prepare_cluster_pairs();
void launch_cluster_pairs(const DevSys& s, const Params& p, int step_off, int part, int list, cudaStream_t st);
void launch_cluster_collect(const DevSys& s, double* out, cudaStream_t st);
// All-pairs tiles (tile.cu): the pair sums of `part` into the atom-indexed
// accumulators, and their read-out (added to out[3n], accumulators cleared).
void launch_tile_pairs(const DevSys& s, const Params& p, int step_off, int part, cudaStream_t st);
void launch_tile_collect(const DevSys& s, double* out, cudaStream_t st);
