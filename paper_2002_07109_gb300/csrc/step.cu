// Fused per-step kernels of BOUNCE (B J A O A J B, paper Sec. III.C and the
// algorithm of Sec. IV.B) and BAOAB.
//
// Step fusion: B and J do not commute, but the end of step n (J then B/2)
// and the start of step n+1 (B/2 then J) act at the same positions.  So one
// step-kernel launch per step does, for every atom, at positions q_n:
//     F_0(q_n)  ->  J(delta/2) [stream 2, step n-1]  ->  B(delta)
//               ->  J(delta/2) [stream 1, step n]   ->  A(delta/2) O A(delta/2)
// writing q_{n+1} to the other position buffer (J of atom i reads partners
// at q_n).  A run is a head launch (B/2 instead of J B), bodies, and a tail
// launch (J then B/2, no drift).  Where F_0's pair sums run over the long
// candidate rows they come from k_pairs, a kernel of their own launched just
// before (more warps in flight on the partners' gathers); short-row pair sums
// stay in the step kernel.
//
// Work mapping (one CTA = 32 consecutive atoms, NW warps):
//   * pair sums and jump proposals are warp-cooperative, lanes over
//     neighbours / proposals, warps over the CTA's atoms;
//   * every FP64 operation (B, A, O, ||v||, Poisson means, accumulation of
//     the jump increments) runs lane-parallel in warp 0, one atom per lane:
//     an FP64 warp instruction costs the same with 1 or 32 active lanes on
//     this GPU, so per-atom FP64 work is never done one lane at a time.
// Jump step of atom i (Sec. IV.B): M ~ Poisson(n_i beta ||v_i|| L* delta/2);
// proposal k draws J (partner) and U from Philox slot k; accept iff
// U ||v_i|| L* < v_i . F_iJ.  The warp evaluates 32 proposals at once with
// the current velocity, takes the first accepted one, reflects, and
// re-evaluates the remaining proposals with the new velocity: the same
// decisions as the sequential loop.  Decisions are screened in FP32 with a
// rigorous error margin and settled in FP64 when inside it; reflections are
// FP32 and their increments are added to the FP64 velocity once per J.
#include "common.cuh"

namespace {

constexpr int NW = 8;  // warps per CTA
static_assert(BOUNCE_GROUP <= 32, "per-atom prefixes are one warp scan");

// Inclusive prefix sum over the 32 lanes of a warp.
__device__ __forceinline__ int warp_scan_incl(int x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}
constexpr int FU = 2;  // proposals per thread in flight in the jump phase
// The staged proposals carry the partner's type group in the low bits of x2
// (x2 & 3), below the 26 bits that u53 reads: room for 4 types.
static_assert(BOUNCE_MAXT <= 4, "the partner type group is packed into 2 bits of x2");

struct JumpSmem {
    double s[BOUNCE_GROUP];       // ||v|| (FP64)
    float sl[BOUNCE_GROUP];       // ||v|| L* (FP32)
    float slt[BOUNCE_GROUP][BOUNCE_MAXT];  // ||v|| times the bound of each partner type (FP32)
    float vf[BOUNCE_GROUP][3];    // FP32 velocity at the start of the chain
    float dv[BOUNCE_GROUP][3];    // accumulated jump increment
    float muc[BOUNCE_GROUP];      // Poisson chunk mean (FP32)
    int nch[BOUNCE_GROUP];        // number of Poisson chunks
    int M[BOUNCE_GROUP];          // proposals of each atom (sum of its Poisson chunks)
    int nacc[BOUNCE_GROUP];
    int chp[BOUNCE_GROUP + 1];    // prefix of the chunk counts
    float inv[129];               // 1/k, k = 0..128 (round-to-nearest reciprocals)
    unsigned long long cnt[3];    // proposals, accepts, near ties
};

// Split FP32 copy (hi, lo) of the position x - of: the slot copies of the
// cluster lists keep the image of the last build (continuous motion across
// faces), whatever the wrap of phi.
__device__ __forceinline__ void split_pos(double x, double y, double z, double ox, double oy, double oz, float w_hi,
                                          float w_lo, float4& ph, float4& pl) {
    const double a = x - ox, b = y - oy, c = z - oz;
    const float hx = __double2float_rn(a), hy = __double2float_rn(b), hz = __double2float_rn(c);
    ph = make_float4(hx, hy, hz, w_hi);
    pl = make_float4(__double2float_rn(a - (double)hx), __double2float_rn(b - (double)hy),
                     __double2float_rn(c - (double)hz), w_lo);
}

// Lane-parallel (warp 0): quantities of the jump step of atom `a` that need FP64.
__device__ __forceinline__ void jump_prep(const DevSys& s, const Params& p, JumpSmem& js, int a, int i, double vx,
                                          double vy, double vz) {
    const double sp = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(vx, vx), __dmul_rn(vy, vy)), __dmul_rn(vz, vz)));
    const int t = s.type[i];
    const double Ls = p.Lstar_d[t];
    // candidates: n_i, or with per-type-pair bounds the row weight W_i 2^-16
    // (W_i = sum_b n_ib Lq_ab, exact in FP64)
    double n;
    if (p.typed) {
        uint32_t W = 0u;
        for (int b = 0; b < BOUNCE_MAXT; ++b) {
            const double lt = p.lt_d[t * BOUNCE_MAXT + b];
            W += (uint32_t)s.nseg[(size_t)i * BOUNCE_MAXT + b] * p.lq[t * BOUNCE_MAXT + b];
            js.slt[a][b] = __double2float_rn(__dmul_rn(sp, lt));
        }
        n = __dmul_rn((double)W, 1.52587890625e-05);
    } else {
        n = (double)s.nlong[i];
    }
    double mu = __dmul_rn(__dmul_rn(__dmul_rn(__dmul_rn(__dmul_rn(p.beta, sp), Ls), n), p.dt), 0.5);
    if (!(mu <= 1e6)) {  // a blown-up state: report instead of drawing millions of proposals
        atomicOr(s.err, BERR_RATE);
        mu = 0.0;
    }
    int nch = 0;
    float muc = 0.f;
    if (mu > 0.0) {
        nch = (int)ceil(__dmul_rn(mu, 0.0625));  // mu / 16, exact
        muc = __double2float_rn(nch == 1 ? mu : __ddiv_rn(mu, (double)nch));
    }
    js.s[a] = sp;
    js.sl[a] = __double2float_rn(__dmul_rn(sp, Ls));
    if (!p.typed) js.slt[a][0] = js.sl[a];
    js.vf[a][0] = __double2float_rn(vx);
    js.vf[a][1] = __double2float_rn(vy);
    js.vf[a][2] = __double2float_rn(vz);
    js.muc[a] = muc;
    js.nch[a] = nch;
}

// Exact FP64 decision U ||v|| L* < v . F for the inputs of one proposal (the
// FP32 screen could not decide it).  Kept out of line so the compiler does
// not hoist its FP64 work into the common path.
__device__ __noinline__ int exact_decision(float vx, float vy, float vz, float gx, float gy, float gz, uint32_t x1,
                                           uint32_t x2, double sp, double Ls) {
    const double ad = __dadd_rn(__dadd_rn(__dmul_rn((double)vx, (double)gx), __dmul_rn((double)vy, (double)gy)),
                                __dmul_rn((double)vz, (double)gz));
    const double td = __dmul_rn(__dmul_rn(u53(x1, x2), sp), Ls);
    return td < ad ? 1 : 0;
}

// Poisson(mu_c) by sequential search of the FP32 CDF with uniform u (same
// operations as poisson_invert_f32); inv[k] = 1/k.
__device__ __forceinline__ int poisson_chunk(float u, float mu_c, const float* inv) {
    float pk = expneg_f32(mu_c), cdf = pk;
    int k = 0;
    while (u > cdf && k < 128) {
        ++k;
        const float q = __fmul_rn(__fmul_rn(pk, mu_c), inv[k]);
        const float cn = __fadd_rn(cdf, q);
        if (cn == cdf) break;
        pk = q;
        cdf = cn;
    }
    return k;
}

// Poisson counts of the CTA's atoms (one half step): every thread takes
// whole chunks (chunk c of atom a inverts Poisson(mu_c) with the uniform of
// Philox slot 0x80000000 | c), one chunk per thread at a time, and adds its
// count to the atom's total.  Called by all threads of the CTA.
__device__ void poisson_phase(const DevSys& s, const Params& p, JumpSmem& js, int base, int na, long long step,
                              uint32_t stream, const float* u0 = nullptr) {
    // every atom with at most one chunk (mu <= 16, the usual case): lane a of
    // warp 0 inverts atom a's chunk, and the prefix scan of jump_phase (same
    // warp) follows without a CTA barrier.  Every warp takes this decision
    // from the chunk counts, which a barrier has published.
    const int lane = threadIdx.x & 31;
    if (__all_sync(0xffffffffu, lane >= na || js.nch[lane] <= 1)) {
        if (threadIdx.x < na) {
            int k = 0;
            if (js.nch[lane] == 1) {
                // u0: the uniforms of chunk 0, drawn ahead by another warp
                const float u = u0 ? u0[lane] : u24(rng_atom(s, p, BOUNCE_POISSON_SLOT, base + lane, step, stream).x);
                k = poisson_chunk(u, js.muc[lane], js.inv);
            }
            js.M[lane] = k;
        }
        __syncwarp();
        return;
    }
    if (threadIdx.x < 32) {  // prefix of the chunk counts: one warp scan (na <= 32)
        const int a = threadIdx.x, c = a < na ? js.nch[a] : 0;
        const int x = warp_scan_incl(c);
        if (a < na) {
            js.chp[a] = x - c;
            js.M[a] = 0;
        }
        if (a == 31) js.chp[na] = x;
    }
    __syncthreads();
    const int tot = js.chp[na];
    for (int t = threadIdx.x; t < tot; t += blockDim.x) {
        int lo = 0, hi = na - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (js.chp[mid] <= t) lo = mid;
            else hi = mid - 1;
        }
        const int c = t - js.chp[lo];
        const uint4 x = rng_atom(s, p, BOUNCE_POISSON_SLOT | (uint32_t)c, base + lo, step, stream);
        atomicAdd(&js.M[lo], poisson_chunk(u24(x.x), js.muc[lo], js.inv));
    }
    __syncthreads();
}

// Proposals staged in shared memory per pass of the jump phase.
constexpr int PC = 2048;

struct PropSmem {
    float gx[PC], gy[PC], gz[PC];  // F_iJ of each staged proposal (zero outside the cutoff)
    uint32_t x1[PC], x2[PC];       // the words that make its uniform U
    int P[BOUNCE_GROUP + 1];       // prefix of the proposal counts M of the CTA's atoms
    float4 ahi[BOUNCE_GROUP], alo[BOUNCE_GROUP];  // the atoms' split positions at q_n
    int an[BOUNCE_GROUP];          // their candidate-row lengths
    uint32_t acum[BOUNCE_GROUP][BOUNCE_MAXT + 1];  // typed rows: cumulative weights C_b (C_T = W_i)
    int ast[BOUNCE_GROUP][BOUNCE_MAXT];    // typed rows: start of each type group
    int alist[BOUNCE_GROUP];       // atoms with proposals in the pass
    int nlist;
    int next;                      // next entry of alist to take in the chain pass
};

// Flattened proposal g of the CTA -> (atom a, slot k = g - P[a] + 1).
__device__ __forceinline__ int owner_of(const PropSmem& ps, int na, int g) {
    int lo = 0, hi = na - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (ps.P[mid] <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// One jump half-step of the CTA's atoms after poisson_phase (Sec. IV.B).
// Passes of up to PC proposals:
// (1) every thread evaluates proposals of the flattened list (the atom's M
//     proposals are contiguous and in slot order), FU at a time so their
//     memory gathers overlap: partner J and U from Philox slot k, and
//     F_iJ = chi W'_sw d / r at q_n, none of which depends on the velocity;
// (2) warps walk the chains: 32 staged proposals at once are decided with the
//     current velocity (accept iff U ||v|| L* < v . F), the first accepted one
//     reflects it, and the rest are decided again with the new velocity --
//     the decisions of the sequential loop.  Decisions are screened in FP32
//     with a rigorous error margin and settled in FP64 inside it.
// The chain velocity (js.vf), its increment (js.dv) and accept count persist
// across passes in shared memory.  Called by all threads of the CTA.
__device__ void jump_phase(const DevSys& s, const Params& p, JumpSmem& js, PropSmem& ps, int cur, int base, int na,
                           long long step, uint32_t stream, bool own_loaded = false) {
    const int lane = threadIdx.x & 31;
    int any = 0;  // the CTA has proposals (warp 0 knows it from the scan)
    if (threadIdx.x < 32) {  // prefix of the proposal counts: one warp scan (na <= 32)
        const int a = threadIdx.x, m = a < na ? js.M[a] : 0;
        const int x = warp_scan_incl(m);
        any = __shfl_sync(0xffffffffu, x, 31) > 0;
        if (a < na) ps.P[a] = x - m;
        if (a == 31) {
            ps.P[na] = x;
            js.cnt[0] += (unsigned long long)x;
        }
        if (a < na) {
            js.nacc[a] = 0;
            js.dv[a][0] = js.dv[a][1] = js.dv[a][2] = 0.f;
        }
    }
    if (threadIdx.x < na && any) {
        const int a = threadIdx.x, i = base + a;
        if (!own_loaded) {
            ps.ahi[a] = s.phi[cur][i];
            ps.alo[a] = s.plo[cur][i];
            ps.an[a] = s.nlong[i];
        }
        if (p.typed) {
            const int ta = s.type[i];
            uint32_t c = 0u;
            int st = 0;
            for (int b = 0; b < BOUNCE_MAXT; ++b) {
                const int nb = s.nseg[(size_t)i * BOUNCE_MAXT + b];
                ps.acum[a][b] = c;
                ps.ast[a][b] = st;
                c += (uint32_t)nb * p.lq[ta * BOUNCE_MAXT + b];
                st += nb;
            }
            ps.acum[a][BOUNCE_MAXT] = c;
        }
    }
    __syncthreads();
    const int tot = ps.P[na];
    if (tot == 0) return;  // no proposals: the velocity increments stay zero
    int near = 0;
    for (int c0 = 0; c0 < tot; c0 += PC) {
        const int cn = min(PC, tot - c0);
        for (int t0 = threadIdx.x; t0 < cn; t0 += FU * NW * 32) {
            int ow[FU], jj[FU];
#pragma unroll
            for (int u = 0; u < FU; ++u) {
                const int t = t0 + u * NW * 32;
                ow[u] = 0;
                jj[u] = -1;
                if (t < cn) {
                    const int g = c0 + t;
                    ow[u] = owner_of(ps, na, g);
                    const uint4 x = rng_atom(s, p, (uint32_t)(g - ps.P[ow[u]] + 1), base + ow[u], step, stream);
                    uint32_t bsel = 0u;
                    if (p.typed) {
                        // two-stage choice: weight unit tg of W_i; its type group b is the
                        // last with C_b <= tg (never an empty group); its member (tg - C_b) / Lq_ab
                        const int a = ow[u], ta = type_of(ps.alo[a]);
                        const uint32_t tg = __umulhi(x.x, ps.acum[a][BOUNCE_MAXT]);
#pragma unroll
                        for (int b = 1; b < BOUNCE_MAXT; ++b)
                            if (ps.acum[a][b] <= tg) bsel = (uint32_t)b;
                        const uint32_t x = tg - ps.acum[a][bsel], ab = ta * BOUNCE_MAXT + bsel;
                        const uint32_t th = __umulhi(p.lq_m[ab], x);
                        jj[u] = ps.ast[a][bsel] + (int)((th + ((x - th) >> 1)) >> p.lq_s[ab]);  // x / Lq_ab
                    } else {
                        jj[u] = (int)__umulhi(x.x, (uint32_t)ps.an[ow[u]]);
                    }
                    ps.x1[t] = x.y;
                    ps.x2[t] = (x.z & ~63u) | bsel;  // u53 uses only the top 26 bits of x2
                }
            }
#pragma unroll
            for (int u = 0; u < FU; ++u)
                if (jj[u] >= 0) jj[u] = s.rows[(size_t)(base + ow[u]) * s.cap + jj[u]];
            float4 hj[FU], lj[FU];
#pragma unroll
            for (int u = 0; u < FU; ++u)
                if (jj[u] >= 0) {
                    hj[u] = s.phi[cur][jj[u]];
                    lj[u] = s.plo[cur][jj[u]];
                }
#pragma unroll
            for (int u = 0; u < FU; ++u) {
                if (jj[u] < 0) continue;
                const int t = t0 + u * NW * 32;
                const float4 hi = ps.ahi[ow[u]], lo = ps.alo[ow[u]];
                const float3 d = pair_disp(p, hi, lo, hj[u], lj[u]);
                const float r2 = d.x * d.x + d.y * d.y + d.z * d.z;
                float gx = 0.f, gy = 0.f, gz = 0.f;
                if (inside_cut(s, p, cur, base + ow[u], jj[u], r2)) {
                    float sw, fixed, r;
                    pair_dW_split(p, r2, p.kcoul * hi.w * hj[u].w, type_of(lo) * BOUNCE_MAXT + type_of(lj[u]), sw,
                                  fixed, r);
                    const float w = chi_of(p, r) * sw;
                    gx = w * d.x;
                    gy = w * d.y;
                    gz = w * d.z;
                }
                ps.gx[t] = gx;
                ps.gy[t] = gy;
                ps.gz[t] = gz;
            }
        }
        if (threadIdx.x < 32) {  // the atoms with proposals in this pass, in order
            const int a = threadIdx.x;
            const bool has = a < na && max(ps.P[a], c0) < min(ps.P[a + 1], c0 + cn);
            const unsigned b = __ballot_sync(0xffffffffu, has);
            if (has) ps.alist[__popc(b & ((1u << a) - 1u))] = a;
            if (a == 0) {
                ps.nlist = __popc(b);
                ps.next = 0;
            }
        }
        __syncthreads();
        for (;;) {
            int k = 0;
            if (lane == 0) k = atomicAdd(&ps.next, 1);
            k = __shfl_sync(0xffffffffu, k, 0);
            if (k >= ps.nlist) break;
            const int a = ps.alist[k];
            const int lo = max(ps.P[a], c0), hi = min(ps.P[a + 1], c0 + cn);
            const int ti = s.type[base + a];
            const double sp = js.s[a];
            const float sp_f = __double2float_rn(sp);
            float vx = js.vf[a][0], vy = js.vf[a][1], vz = js.vf[a][2];
            float dvx = js.dv[a][0], dvy = js.dv[a][1], dvz = js.dv[a][2];
            int nacc = js.nacc[a];
            for (int gb = lo; gb < hi; gb += 32) {
                const int t = gb - c0 + lane;
                const bool act = gb + lane < hi;
                float gx = 0.f, gy = 0.f, gz = 0.f, g2 = 1.f, thr = 0.f, hi = 0.f, lo = 0.f, tie = 0.f;
                uint32_t x1 = 0, x2 = 0;
                if (act) {
                    gx = ps.gx[t];
                    gy = ps.gy[t];
                    gz = ps.gz[t];
                    x1 = ps.x1[t];
                    x2 = ps.x2[t];
                    const float sl = js.slt[a][x2 & 3u];  // ||v|| times the bound of the partner's type
                    thr = u24(x1) * sl;
                    g2 = gx * gx + gy * gy + gz * gz;
                    // FP32 decision error: |fl(v.F) - v.F| <= 4e-6 sum_c |v_c F_c| <= 4e-6 ||v|| ||F||
                    // (the chain's FP32 ||v|| stays within 1e-4 of the FP64 one, reflections keep it);
                    // U and ||v|| L within 2.4e-7 ||v|| L.  Fixed along the chain.
                    const float err = 4e-6f * (thr + 1.0001f * sp_f * sqrtf(g2)) + 2.4e-7f * sl;
                    hi = thr + err;
                    lo = thr - err;
                    tie = 1e-6f * sl;
                }
                int start = 0;
                while (true) {
                    // decide with the current velocity: accept iff U ||v|| L < v . F
                    const float af = vx * gx + vy * gy + vz * gz;
                    int dec = (hi < af) ? 1 : ((lo > af) ? 0 : 2);
                    const bool live = act && lane >= start;
                    if (__any_sync(0xffffffffu, live && dec == 2)) {
                        if (live && dec == 2) {
                            const double Ls = p.typed ? p.lt_d[ti * BOUNCE_MAXT + (x2 & 3u)] : p.Lstar_d[ti];
                            dec = exact_decision(vx, vy, vz, gx, gy, gz, x1, x2, sp, Ls);
                        }
                    }
                    const uint32_t acc = __ballot_sync(0xffffffffu, live && dec == 1);
                    const int f = acc ? __ffs(acc) - 1 : 32;
                    // near ties among the decisions that stand (lanes start..f)
                    if (live && lane <= f && fabsf(thr - af) < tie) ++near;
                    if (!acc) break;
                    // reflect on the accepted proposal: its v.F and ||F||^2 from its lane
                    const float fx = __shfl_sync(0xffffffffu, gx, f), fy = __shfl_sync(0xffffffffu, gy, f),
                                fz = __shfl_sync(0xffffffffu, gz, f);
                    const float aa = __shfl_sync(0xffffffffu, af, f), ff = __shfl_sync(0xffffffffu, g2, f);
                    const float coef = __fdividef(aa + aa, ff);
                    vx -= coef * fx;
                    vy -= coef * fy;
                    vz -= coef * fz;
                    dvx -= coef * fx;
                    dvy -= coef * fy;
                    dvz -= coef * fz;
                    ++nacc;
                    start = f + 1;
                }
            }
            if (lane == 0) {
                js.vf[a][0] = vx;
                js.vf[a][1] = vy;
                js.vf[a][2] = vz;
                js.dv[a][0] = dvx;
                js.dv[a][1] = dvy;
                js.dv[a][2] = dvz;
                js.nacc[a] = nacc;
            }
        }
        __syncthreads();
    }
    near = warp_sum_i(near);
    if (lane == 0 && near) atomicAdd(&js.cnt[2], (unsigned long long)near);
    if (threadIdx.x < 32) {
        const int A = warp_sum_i(threadIdx.x < na ? js.nacc[threadIdx.x] : 0);
        if (threadIdx.x == 0) js.cnt[1] += (unsigned long long)A;
    }
    __syncthreads();
}

// Warp-cooperative gradient of atom i: part 0 = full (long rows, chi = 1),
// 1 = short (short rows, 1 - chi), 2 = long (long rows, chi), 3 = short
// pairs without bonded terms, 4 = bonded terms only, 5 = full pairs without
// bonded terms; bonded terms are added for parts 0, 1 and 4.
__device__ float3 atom_gradient(const DevSys& s, const Params& p, int cur, int i, int part, int& npairs) {
    const int lane = threadIdx.x & 31;
    const float4 hi = s.phi[cur][i], lo = s.plo[cur][i];
    const float qi = hi.w;
    const int ti = type_of(lo);
    const bool shortrows = (part == 1 || part == 3) && p.rshort2 < INFINITY;
    const int n = part == 4 ? 0 : (shortrows ? s.nshort[i] : s.nlong[i]);
    const int* row = shortrows ? s.srows + (size_t)i * s.caps : s.rows + (size_t)i * s.cap;
    float gx = 0.f, gy = 0.f, gz = 0.f;
    // software pipeline over the lane's row entries lane, lane + 32, ...: the
    // index two entries ahead and the position one entry ahead are in flight
    // while an entry is evaluated; each lane adds its pairs in row order
    int jc = lane < n ? row[lane] : -1;
    int jn = lane + 32 < n ? row[lane + 32] : -1;
    float4 hc = make_float4(0.f, 0.f, 0.f, 0.f), lc = hc;
    if (jc >= 0) {
        hc = s.phi[cur][jc];
        lc = s.plo[cur][jc];
    }
    for (int k0 = lane; k0 < n; k0 += 32) {
        const int jnn = k0 + 64 < n ? __ldg(row + k0 + 64) : -1;
        float4 hn = hc, ln = lc;
        if (jn >= 0) {
            hn = s.phi[cur][jn];
            ln = s.plo[cur][jn];
        }
        const float3 d = pair_disp(p, hi, lo, hc, lc);
        const float r2 = d.x * d.x + d.y * d.y + d.z * d.z;
        if (inside_cut(s, p, cur, i, jc, r2)) {
            float w;
            if (part == 1 || part == 3) {
                w = pair_dW_f0(p, r2, p.kcoul * qi * hc.w, ti * BOUNCE_MAXT + type_of(lc));
            } else {
                float sw, fixed, r;
                pair_dW_split(p, r2, p.kcoul * qi * hc.w, ti * BOUNCE_MAXT + type_of(lc), sw, fixed, r);
                w = part == 2 ? sw * chi_of(p, r) : sw + fixed;
            }
            gx += w * d.x;
            gy += w * d.y;
            gz += w * d.z;
        }
        jc = jn;
        jn = jnn;
        hc = hn;
        lc = ln;
    }
    if (part == 0 || part == 1 || part == 4) {
        for (int t = s.bt_off[i] + lane; t < s.bt_off[i + 1]; t += 32) {
            const float3 g = bonded_grad(p, s, cur, i, s.bt_idx[t], s.bt_par[t]);
            gx += g.x;
            gy += g.y;
            gz += g.z;
        }
    }
    npairs = n;
    return make_float3(warp_sum_f(gx), warp_sum_f(gy), warp_sum_f(gz));
}

// variant: 0 head (B/2 [J1] A O A), 1 body ([J2] B [J1] A O A), 2 tail ([J2] B/2)
// hr: time over which the reciprocal-space gradient kicks at this boundary
// (0 without it; delta or delta/2 when it is part of F_0 or of BAOAB's full
// gradient; Delta or Delta/2 at BOUNCE-RESPA block boundaries).
// ext: the extended RESPA split -- F_0 holds only the bonded terms and the
// short-range pair part kicks over hout (Delta or Delta/2 at block
// boundaries, 0 elsewhere, where the pair sums are skipped).
template <int BOUNCE>
__global__ void __launch_bounds__(NW * 32, 3) k_step(DevSys s, Params p, int variant, int step_off, double hr,
                                                     int ext, double hout, int pre) {
    __shared__ float sG[BOUNCE_GROUP][3];
    __shared__ float sGp[BOUNCE_GROUP][3];
    __shared__ double sV[BOUNCE_GROUP][3];
    __shared__ JumpSmem js;
    __shared__ PropSmem ps;
    __shared__ int sBoff[BOUNCE_GROUP + 1];
    __shared__ unsigned long long sPairs;
    // per-atom inputs of warp 0's FP64 phases, fetched ahead by warps 1-4
    __shared__ double sQ[BOUNCE_GROUP][3], sRef[BOUNCE_GROUP][3], sKick[BOUNCE_GROUP], sOsd[BOUNCE_GROUP];
    __shared__ double sCref[BOUNCE_GROUP][3];
    __shared__ int sSlot[BOUNCE_GROUP];
    __shared__ float sNz[BOUNCE_GROUP][3], sU[2][BOUNCE_GROUP], sHw[BOUNCE_GROUP], sLw[BOUNCE_GROUP];
    chain_enter();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int base = blockIdx.x * BOUNCE_GROUP;
    const int na = min(BOUNCE_GROUP, s.n - base);
    const long long step = *s.step_base + step_off;
    const int cur = (int)(step & 1), nxt = cur ^ 1;
    const bool do_j2 = BOUNCE && variant != 0;
    const bool do_j1 = BOUNCE && variant != 2;
    const bool do_aoa = variant != 2;
    const double hk = variant == 1 ? p.dt : 0.5 * p.dt;
    if (threadIdx.x == 0) {
        sPairs = 0ull;
        js.cnt[0] = js.cnt[1] = js.cnt[2] = 0ull;
    }
    if (BOUNCE)
        for (int k = threadIdx.x; k < 129; k += blockDim.x) js.inv[k] = k ? __frcp_rn((float)k) : 0.f;
    if (threadIdx.x <= na) sBoff[threadIdx.x] = s.bt_off[base + threadIdx.x];
    __syncthreads();
    // warps 1-4 fetch ahead what warp 0's FP64 phases read (own positions,
    // kick and O-step factors, the O-step and Poisson draws), so that warp 0's
    // critical path waits on shared memory, not on global loads or Philox
    if (warp >= 1 && warp <= 4 && lane < na) {
        const int i = base + lane;
        if (warp == 1 && do_aoa) {  // O: Box-Muller on Philox slot 0, stream 0
            const uint4 r = rng_atom(s, p, 0u, i, step, BOUNCE_STREAM_O);
            const float ra = sqrtf(-2.f * logf(u24_open0(r.x)));
            float sn, cs;
            sincospif(2.f * u24(r.y), &sn, &cs);
            sNz[lane][0] = ra * cs;
            sNz[lane][1] = ra * sn;
            sNz[lane][2] = sqrtf(-2.f * logf(u24_open0(r.z))) * cospif(2.f * u24(r.w));
        } else if (warp == 2 && BOUNCE) {  // chunk 0 of each jump half-step's Poisson count
            if (do_j2) sU[0][lane] = u24(rng_atom(s, p, BOUNCE_POISSON_SLOT, i, step - 1, BOUNCE_STREAM_J2).x);
            if (do_j1) sU[1][lane] = u24(rng_atom(s, p, BOUNCE_POISSON_SLOT, i, step, BOUNCE_STREAM_J1).x);
        } else if (warp == 3) {
            sQ[lane][0] = s.qx[cur][i];
            sQ[lane][1] = s.qy[cur][i];
            sQ[lane][2] = s.qz[cur][i];
            sKick[lane] = s.kick[i];
            if (do_aoa) {
                sOsd[lane] = s.osd[i];
                sRef[lane][0] = s.refx[i];
                sRef[lane][1] = s.refy[i];
                sRef[lane][2] = s.refz[i];
                if (s.cl.on) {
                    sCref[lane][0] = s.cl.crefx[i];
                    sCref[lane][1] = s.cl.crefy[i];
                    sCref[lane][2] = s.cl.crefz[i];
                }
            }
        } else if (warp == 4) {
            const float4 h = s.phi[cur][i], l = s.plo[cur][i];
            sHw[lane] = h.w;
            sLw[lane] = l.w;
            if (BOUNCE) {
                ps.ahi[lane] = h;
                ps.alo[lane] = l;
                ps.an[lane] = s.nlong[i];
            }
        }
    }
    // F_0 (BOUNCE) or the full gradient (BAOAB) at q_n: pair sums, either
    // read from k_pairs (pre) or here, warps over atoms
    if (pre && threadIdx.x < na) {
        const int a = threadIdx.x, i = base + a;
        float4 g;
        if (s.cl.on || s.tl.on) {
            // cluster or tile pair sums: the atom's fixed-point accumulators
            // (by slot, or by atom), cleared for the next evaluation
            const int sl = s.cl.on ? s.cl.a2s[i] : i;
            sSlot[a] = sl;
            const size_t ns = s.cl.on ? (size_t)s.cl.ncol * s.cl.maxcl * BOUNCE_CL : (size_t)s.n;
            unsigned long long* acc = s.cl.on ? s.cl.acc : s.tl.acc;
            g = make_float4((float)((double)(long long)acc[sl] * CL_UNFIX),
                            (float)((double)(long long)acc[ns + sl] * CL_UNFIX),
                            (float)((double)(long long)acc[2 * ns + sl] * CL_UNFIX), 0.f);
            acc[sl] = 0ull;
            acc[ns + sl] = 0ull;
            acc[2 * ns + sl] = 0ull;
        } else {
            g = s.g0[i];
            atomicAdd(&sPairs, (unsigned long long)__float_as_int(g.w));
        }
        const bool to_out = ext != 0;
        sG[a][0] = to_out ? 0.f : g.x;
        sG[a][1] = to_out ? 0.f : g.y;
        sG[a][2] = to_out ? 0.f : g.z;
        sGp[a][0] = to_out ? g.x : 0.f;
        sGp[a][1] = to_out ? g.y : 0.f;
        sGp[a][2] = to_out ? g.z : 0.f;
    } else if (s.cl.on && do_aoa && threadIdx.x < na) {
        sSlot[threadIdx.x] = s.cl.a2s[base + threadIdx.x];
    }
    for (int a = pre ? na : warp; a < na; a += NW) {
        int np = 0, np2 = 0;
        float3 g = make_float3(0.f, 0.f, 0.f), gp = g;
        if (!ext) g = atom_gradient(s, p, cur, base + a, BOUNCE ? 3 : 5, np);
        if (ext && hout != 0.0) gp = atom_gradient(s, p, cur, base + a, 3, np2);
        if (lane == 0) {
            sG[a][0] = g.x;
            sG[a][1] = g.y;
            sG[a][2] = g.z;
            sGp[a][0] = gp.x;
            sGp[a][1] = gp.y;
            sGp[a][2] = gp.z;
            atomicAdd(&sPairs, (unsigned long long)(np + np2));
        }
    }
    // bonded terms: one term per thread into the staging area, then each atom
    // adds its own terms in list order (lane a of warp 0)
    {
        const int e0 = sBoff[0], e1 = sBoff[na];
        for (int c = e0; c < e1; c += NW * 32) {
            const int e = c + threadIdx.x;
            if (e < e1) {
                int lo = 0, hi = na - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (sBoff[mid] <= e) lo = mid;
                    else hi = mid - 1;
                }
                const float3 g = bonded_grad(p, s, cur, base + lo, s.bt_idx[e], s.bt_par[e]);
                ps.gx[threadIdx.x] = g.x;
                ps.gy[threadIdx.x] = g.y;
                ps.gz[threadIdx.x] = g.z;
            }
            __syncthreads();
            if (warp == 0 && lane < na) {
                const int t0 = max(sBoff[lane], c), t1 = min(sBoff[lane + 1], c + NW * 32);
                float bx = 0.f, by = 0.f, bz = 0.f;
                for (int t = t0; t < t1; ++t) {
                    bx += ps.gx[t - c];
                    by += ps.gy[t - c];
                    bz += ps.gz[t - c];
                }
                sG[lane][0] += bx;
                sG[lane][1] += by;
                sG[lane][2] += bz;
            }
            __syncthreads();
        }
    }
    if (warp == 0 && lane < na) {
        const int i = base + lane;
        const double vx = s.vx[i], vy = s.vy[i], vz = s.vz[i];
        sV[lane][0] = vx;
        sV[lane][1] = vy;
        sV[lane][2] = vz;
        if (do_j2) jump_prep(s, p, js, lane, i, vx, vy, vz);
    }
    __syncthreads();
    if (do_j2) {
        poisson_phase(s, p, js, base, na, step - 1, BOUNCE_STREAM_J2, sU[0]);
        jump_phase(s, p, js, ps, cur, base, na, step - 1, BOUNCE_STREAM_J2, true);
    }
    if (warp == 0 && lane < na) {
        const int i = base + lane;
        double vx = sV[lane][0], vy = sV[lane][1], vz = sV[lane][2];
        if (do_j2) {
            vx += (double)js.dv[lane][0];
            vy += (double)js.dv[lane][1];
            vz += (double)js.dv[lane][2];
        }
        const double c = hk * sKick[lane];
        vx -= c * (double)sG[lane][0];
        vy -= c * (double)sG[lane][1];
        vz -= c * (double)sG[lane][2];
        if (hr != 0.0) {
            const double cr = hr * sKick[lane];
            vx -= cr * s.grecip[i];
            vy -= cr * s.grecip[s.n + i];
            vz -= cr * s.grecip[2 * (size_t)s.n + i];
        }
        if (ext && hout != 0.0) {
            const double co = hout * sKick[lane];
            vx -= co * (double)sGp[lane][0];
            vy -= co * (double)sGp[lane][1];
            vz -= co * (double)sGp[lane][2];
        }
        sV[lane][0] = vx;
        sV[lane][1] = vy;
        sV[lane][2] = vz;
        if (do_j1) jump_prep(s, p, js, lane, i, vx, vy, vz);
    }
    __syncthreads();
    if (do_j1) {
        poisson_phase(s, p, js, base, na, step, BOUNCE_STREAM_J1, sU[1]);
        jump_phase(s, p, js, ps, cur, base, na, step, BOUNCE_STREAM_J1, true);
    }
    if (warp == 0 && lane < na) {
        const int i = base + lane;
        double vx = sV[lane][0], vy = sV[lane][1], vz = sV[lane][2];
        if (do_j1) {
            vx += (double)js.dv[lane][0];
            vy += (double)js.dv[lane][1];
            vz += (double)js.dv[lane][2];
        }
        if (do_aoa) {
            const double h = 0.5 * p.dt;
            double x = sQ[lane][0] + h * vx, y = sQ[lane][1] + h * vy, z = sQ[lane][2] + h * vz;
            // O: the Box-Muller normals drawn ahead (Philox slot 0, stream 0)
            const double sd = sOsd[lane];
            vx = p.c1 * vx + sd * (double)sNz[lane][0];
            vy = p.c1 * vy + sd * (double)sNz[lane][1];
            vz = p.c1 * vz + sd * (double)sNz[lane][2];
            x += h * vx;
            y += h * vy;
            z += h * vz;
            s.qx[nxt][i] = x;
            s.qy[nxt][i] = y;
            s.qz[nxt][i] = z;
            double wx = x, wy = y, wz = z;
            if (p.periodic) {
                wx = wrap_box(x, p.Ld[0], p.iLd[0]);
                wy = wrap_box(y, p.Ld[1], p.iLd[1]);
                wz = wrap_box(z, p.Ld[2], p.iLd[2]);
            }
            const float hx = __double2float_rn(wx), hy = __double2float_rn(wy), hz = __double2float_rn(wz);
            const float4 ph = make_float4(hx, hy, hz, sHw[lane]);
            const float4 pl = make_float4(__double2float_rn(wx - (double)hx), __double2float_rn(wy - (double)hy),
                                          __double2float_rn(wz - (double)hz), sLw[lane]);
            s.phi[nxt][i] = ph;
            s.plo[nxt][i] = pl;
            const double ex = x - sRef[lane][0], ey = y - sRef[lane][1], ez = z - sRef[lane][2];
            if (s.rows_flag && ((s.rows_move >> __float_as_int(sLw[lane])) & 1) &&
                ex * ex + ey * ey + ez * ez > p.skin_half2)
                atomicOr(s.rebuild, 1);
            if (s.cl.on) {
                // slot-ordered copy for the cluster pair kernel (in the image of the
                // build); displacement since the cluster build
                const int sl = sSlot[lane];
                float4 ch = ph, cw = pl;
                if (p.periodic) split_pos(x, y, z, s.cl.cofx[i], s.cl.cofy[i], s.cl.cofz[i], ph.w, pl.w, ch, cw);
                s.cl.sphi[nxt][sl] = ch;
                s.cl.splo[nxt][sl] = cw;
                const double cx = x - sCref[lane][0], cy = y - sCref[lane][1], cz = z - sCref[lane][2];
                if (cx * cx + cy * cy + cz * cz > s.cl.cskin_half2) atomicOr(s.cl.rebuild, 1);
                // displacement since the last prune of the lists
                const float4 pr = s.cl.pref[sl];
                const float px = ch.x - pr.x, py = ch.y - pr.y, pz = ch.z - pr.z;
                if (px * px + py * py + pz * pz > s.cl.pdisp2) atomicOr(s.cl.prune, 1);
            }
        }
        s.vx[i] = vx;
        s.vy[i] = vy;
        s.vz[i] = vz;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicAdd(&s.cnt[BOUNCE ? CNT_SHORT_PAIRS : CNT_FULL_PAIRS], sPairs);
        if (BOUNCE) {
            atomicAdd(&s.cnt[CNT_PROPOSALS], js.cnt[0]);
            atomicAdd(&s.cnt[CNT_ACCEPTS], js.cnt[1]);
            atomicAdd(&s.cnt[CNT_NEAR], js.cnt[2]);
        }
    }
}

// ---------------------------------------------------------------- lite step
// The same step as k_step with one thread per atom and no CTA barriers, for
// runs whose jump proposals are rare (BAOAB, or BOUNCE splits with well
// under one proposal per atom-step): each thread takes its atom's pair sums
// from the pair kernel, adds its bonded terms in list order, and runs the
// two jump half-steps of its atom sequentially -- the Poisson chunks, then
// proposal k = 1..M in order, each decided with the velocity left by the
// proposals before it -- with the arithmetic of jump_prep, poisson_phase
// and jump_phase, so both kernels give the same results bit for bit.

// One jump half-step J(delta/2) of atom i (thread-sequential): returns the
// FP32 velocity increment and counts proposals, accepts and near ties.
__device__ __forceinline__ void jump_thread(const DevSys& s, const Params& p, int cur, int i, int ti, double vx,
                                            double vy, double vz, long long step, uint32_t stream, float4 ahi,
                                            float4 alo, float& dvx, float& dvy, float& dvz, int& nprop, int& nacc,
                                            int& near) {
    dvx = dvy = dvz = 0.f;
    const double Ls = p.Lstar_d[ti];
    if (Ls == 0.0) return;  // no jump part for this type: Poisson mean 0 (skips the FP64 set-up)
    if (!p.typed) {
        // Most atoms draw no proposal.  An FP32 upper bound mu_f of the mean
        // (every rounding covered by the factor 1 + 1e-5) and the same first
        // Poisson draw settle M = 0 without the FP64 set-up: expneg_f32 is
        // within 1e-6 of exp(-x), so u <= expneg_f32(mu_f) (1 - 4e-6) implies
        // u <= expneg_f32(float(mu)), which is the exact path's M = 0.
        const float fx = __double2float_rn(vx), fy = __double2float_rn(vy), fz = __double2float_rn(vz);
        const float spf = sqrtf(fx * fx + fy * fy + fz * fz);
        const float muf = p.beta_f * spf * p.Lstar_f[ti] * (float)s.nlong[i] * p.dt_half_f * 1.00001f;
        if (muf < 1.f) {
            const float u = u24(rng_atom(s, p, BOUNCE_POISSON_SLOT, i, step, stream).x);
            if (u <= __fmul_rn(expneg_f32(muf), 0.999996f)) return;
        }
    }
    const double sp = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(vx, vx), __dmul_rn(vy, vy)), __dmul_rn(vz, vz)));
    double n;
    uint32_t acum[BOUNCE_MAXT + 1];
    int ast[BOUNCE_MAXT];
    float slt[BOUNCE_MAXT];
    if (p.typed) {
        uint32_t W = 0u;
        int st = 0;
#pragma unroll
        for (int b = 0; b < BOUNCE_MAXT; ++b) {
            const int nb = s.nseg[(size_t)i * BOUNCE_MAXT + b];
            acum[b] = W;
            ast[b] = st;
            W += (uint32_t)nb * p.lq[ti * BOUNCE_MAXT + b];
            st += nb;
            slt[b] = __double2float_rn(__dmul_rn(sp, p.lt_d[ti * BOUNCE_MAXT + b]));
        }
        acum[BOUNCE_MAXT] = W;
        n = __dmul_rn((double)W, 1.52587890625e-05);
    } else {
        n = (double)s.nlong[i];
    }
    double mu = __dmul_rn(__dmul_rn(__dmul_rn(__dmul_rn(__dmul_rn(p.beta, sp), Ls), n), p.dt), 0.5);
    if (!(mu <= 1e6)) {
        atomicOr(s.err, BERR_RATE);
        mu = 0.0;
    }
    if (!(mu > 0.0)) return;
    const int nch = (int)ceil(__dmul_rn(mu, 0.0625));
    const float muc = __double2float_rn(nch == 1 ? mu : __ddiv_rn(mu, (double)nch));
    int M = 0;
    for (int c = 0; c < nch; ++c) {
        const float u = u24(rng_atom(s, p, BOUNCE_POISSON_SLOT | (uint32_t)c, i, step, stream).x);
        float pk = expneg_f32(muc), cdf = pk;
        int k = 0;
        while (u > cdf && k < 128) {
            ++k;
            const float q = __fmul_rn(__fmul_rn(pk, muc), __frcp_rn((float)k));
            const float cn = __fadd_rn(cdf, q);
            if (cn == cdf) break;
            pk = q;
            cdf = cn;
        }
        M += k;
    }
    nprop += M;
    if (M == 0) return;
    const float sl = __double2float_rn(__dmul_rn(sp, Ls));
    if (!p.typed) slt[0] = sl;
    const float sp_f = __double2float_rn(sp);
    float fvx = __double2float_rn(vx), fvy = __double2float_rn(vy), fvz = __double2float_rn(vz);
    const int* row = s.rows + (size_t)i * s.cap;
    const int an = s.nlong[i];
    for (int k = 1; k <= M; ++k) {
        const uint4 x = rng_atom(s, p, (uint32_t)k, i, step, stream);
        uint32_t bsel = 0u;
        int jj;
        if (p.typed) {
            const uint32_t tg = __umulhi(x.x, acum[BOUNCE_MAXT]);
#pragma unroll
            for (int b = 1; b < BOUNCE_MAXT; ++b)
                if (acum[b] <= tg) bsel = (uint32_t)b;
            uint32_t cb = 0u;
            int sb = 0;
#pragma unroll
            for (int b = 0; b < BOUNCE_MAXT; ++b)
                if ((uint32_t)b == bsel) {
                    cb = acum[b];
                    sb = ast[b];
                }
            const uint32_t xx = tg - cb, ab = ti * BOUNCE_MAXT + bsel;
            const uint32_t th = __umulhi(p.lq_m[ab], xx);
            jj = sb + (int)((th + ((xx - th) >> 1)) >> p.lq_s[ab]);
        } else {
            jj = (int)__umulhi(x.x, (uint32_t)an);
        }
        const uint32_t x1 = x.y, x2 = (x.z & ~63u) | bsel;
        const int j = row[jj];
        const float4 hj = s.phi[cur][j], lj = s.plo[cur][j];
        const float3 d = pair_disp(p, ahi, alo, hj, lj);
        const float r2 = d.x * d.x + d.y * d.y + d.z * d.z;
        float gx = 0.f, gy = 0.f, gz = 0.f;
        if (inside_cut(s, p, cur, i, j, r2)) {
            float sw, fixed, r;
            pair_dW_split(p, r2, p.kcoul * ahi.w * hj.w, type_of(alo) * BOUNCE_MAXT + type_of(lj), sw, fixed, r);
            const float w = chi_of(p, r) * sw;
            gx = w * d.x;
            gy = w * d.y;
            gz = w * d.z;
        }
        float slb = slt[0];
#pragma unroll
        for (int b = 1; b < BOUNCE_MAXT; ++b)
            if ((uint32_t)b == (x2 & 3u)) slb = slt[b];
        const float thr = u24(x1) * slb;
        const float g2 = gx * gx + gy * gy + gz * gz;
        const float err = 4e-6f * (thr + 1.0001f * sp_f * sqrtf(g2)) + 2.4e-7f * slb;
        const float af = fvx * gx + fvy * gy + fvz * gz;
        int dec = (thr + err < af) ? 1 : ((thr - err > af) ? 0 : 2);
        if (dec == 2) {
            const double Lb = p.typed ? p.lt_d[ti * BOUNCE_MAXT + (x2 & 3u)] : p.Lstar_d[ti];
            dec = exact_decision(fvx, fvy, fvz, gx, gy, gz, x1, x2, sp, Lb);
        }
        if (fabsf(thr - af) < 1e-6f * slb) ++near;
        if (dec == 1) {
            const float coef = __fdividef(af + af, g2);
            fvx -= coef * gx;
            fvy -= coef * gy;
            fvz -= coef * gz;
            dvx -= coef * gx;
            dvy -= coef * gy;
            dvz -= coef * gz;
            ++nacc;
        }
    }
}

// The jump half-step of atom i in the thread-per-atom kernel: the velocity
// in FP64 registers, updated by the FP32 increment of jump_thread.
__device__ __forceinline__ void jump_lite(const DevSys& s, const Params& p, int cur, int i, long long step,
                                          uint32_t stream, float4 ahi, float4 alo, double& vx, double& vy,
                                          double& vz, int& nprop, int& nacc, int& near) {
    float dx, dy, dz;
    jump_thread(s, p, cur, i, type_of(alo), vx, vy, vz, step, stream, ahi, alo, dx, dy, dz, nprop, nacc, near);
    vx += (double)dx;
    vy += (double)dy;
    vz += (double)dz;
}

// Resident CTAs per SM the thread-per-atom kernel is compiled for: three
// fit the 98,304-atom box's 384 CTAs in one wave (the register cap costs a
// few spills around the jump phases, less than a second wave).
#ifndef LITE_MIN_CTAS
#define LITE_MIN_CTAS 3
#endif

template <int BOUNCE>
__global__ void __launch_bounds__(256, LITE_MIN_CTAS) k_step_lite(DevSys s, Params p, int variant, int step_off,
                                                                  double hr, int ext, double hout) {
    __shared__ unsigned long long cnt[4];
    chain_enter();
    if (threadIdx.x < 4) cnt[threadIdx.x] = 0ull;
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = i < s.n;
    int nprop = 0, nacc = 0, near = 0;
    const long long step = *s.step_base + step_off;
    const int cur = (int)(step & 1), nxt = cur ^ 1;
    const bool do_j2 = BOUNCE && variant != 0;
    const bool do_j1 = BOUNCE && variant != 2;
    const bool do_aoa = variant != 2;
    const double hk = variant == 1 ? p.dt : 0.5 * p.dt;
    __syncthreads();  // the counters are cleared
    // pair sums of the pair kernel (absent between the outer kicks of the extended splits)
    float gx = 0.f, gy = 0.f, gz = 0.f, Gx = 0.f, Gy = 0.f, Gz = 0.f;
    int sl = i;
    float4 ahi = make_float4(0.f, 0.f, 0.f, 0.f), alo = ahi;
    double kick = 0.0, vx = 0.0, vy = 0.0, vz = 0.0;
    if (live) {
        if (s.cl.on) sl = s.cl.a2s[i];
        if (!(ext && hout == 0.0)) {
            const size_t ns = s.cl.on ? (size_t)s.cl.ncol * s.cl.maxcl * BOUNCE_CL : (size_t)s.n;
            unsigned long long* acc = s.cl.on ? s.cl.acc : s.tl.acc;
            gx = (float)((double)(long long)acc[sl] * CL_UNFIX);
            gy = (float)((double)(long long)acc[ns + sl] * CL_UNFIX);
            gz = (float)((double)(long long)acc[2 * ns + sl] * CL_UNFIX);
            acc[sl] = 0ull;
            acc[ns + sl] = 0ull;
            acc[2 * ns + sl] = 0ull;
        }
        Gx = ext ? 0.f : gx;
        Gy = ext ? 0.f : gy;
        Gz = ext ? 0.f : gz;
        // bonded terms of the atom, in list order
        float bx = 0.f, by = 0.f, bz = 0.f;
        for (int t = s.bt_off[i]; t < s.bt_off[i + 1]; ++t) {
            const float3 g = bonded_grad(p, s, cur, i, s.bt_idx[t], s.bt_par[t]);
            bx += g.x;
            by += g.y;
            bz += g.z;
        }
        Gx += bx;
        Gy += by;
        Gz += bz;
        ahi = s.phi[cur][i];
        alo = s.plo[cur][i];
        kick = s.kick[i];
        vx = s.vx[i];
        vy = s.vy[i];
        vz = s.vz[i];
    }
    // the jump half-steps, one thread per atom: most atoms settle M = 0 from
    // their first draw (jump_thread), so no compaction or barrier pays off
    if (do_j2 && live) jump_lite(s, p, cur, i, step - 1, BOUNCE_STREAM_J2, ahi, alo, vx, vy, vz, nprop, nacc, near);
    if (live) {
        const double c = hk * kick;
        vx -= c * (double)Gx;
        vy -= c * (double)Gy;
        vz -= c * (double)Gz;
        if (hr != 0.0) {
            const double cr = hr * kick;
            vx -= cr * s.grecip[i];
            vy -= cr * s.grecip[s.n + i];
            vz -= cr * s.grecip[2 * (size_t)s.n + i];
        }
        if (ext && hout != 0.0) {
            const double co = hout * kick;
            vx -= co * (double)gx;
            vy -= co * (double)gy;
            vz -= co * (double)gz;
        }
    }
    if (do_j1 && live) jump_lite(s, p, cur, i, step, BOUNCE_STREAM_J1, ahi, alo, vx, vy, vz, nprop, nacc, near);
    if (live) {
        if (do_aoa) {
            const double h = 0.5 * p.dt;
            double x = s.qx[cur][i] + h * vx, y = s.qy[cur][i] + h * vy, z = s.qz[cur][i] + h * vz;
            // O: Box-Muller on Philox slot 0, stream 0
            const uint4 r = rng_atom(s, p, 0u, i, step, BOUNCE_STREAM_O);
            const float ra = sqrtf(-2.f * logf(u24_open0(r.x)));
            float sn, cs;
            sincospif(2.f * u24(r.y), &sn, &cs);
            const float n0 = ra * cs, n1 = ra * sn;
            const float n2 = sqrtf(-2.f * logf(u24_open0(r.z))) * cospif(2.f * u24(r.w));
            const double sd = s.osd[i];
            vx = p.c1 * vx + sd * (double)n0;
            vy = p.c1 * vy + sd * (double)n1;
            vz = p.c1 * vz + sd * (double)n2;
            x += h * vx;
            y += h * vy;
            z += h * vz;
            s.qx[nxt][i] = x;
            s.qy[nxt][i] = y;
            s.qz[nxt][i] = z;
            double wx = x, wy = y, wz = z;
            if (p.periodic) {
                wx = wrap_box(x, p.Ld[0], p.iLd[0]);
                wy = wrap_box(y, p.Ld[1], p.iLd[1]);
                wz = wrap_box(z, p.Ld[2], p.iLd[2]);
            }
            const float hx = __double2float_rn(wx), hy = __double2float_rn(wy), hz = __double2float_rn(wz);
            const float4 ph = make_float4(hx, hy, hz, ahi.w);
            const float4 pl = make_float4(__double2float_rn(wx - (double)hx), __double2float_rn(wy - (double)hy),
                                          __double2float_rn(wz - (double)hz), alo.w);
            s.phi[nxt][i] = ph;
            s.plo[nxt][i] = pl;
            const double ex = x - s.refx[i], ey = y - s.refy[i], ez = z - s.refz[i];
            if (s.rows_flag && ((s.rows_move >> type_of(alo)) & 1) && ex * ex + ey * ey + ez * ez > p.skin_half2)
                atomicOr(s.rebuild, 1);
            if (s.cl.on) {
                float4 ch = ph, cw = pl;
                if (p.periodic) split_pos(x, y, z, s.cl.cofx[i], s.cl.cofy[i], s.cl.cofz[i], ph.w, pl.w, ch, cw);
                s.cl.sphi[nxt][sl] = ch;
                s.cl.splo[nxt][sl] = cw;
                const double cx = x - s.cl.crefx[i], cy = y - s.cl.crefy[i], cz = z - s.cl.crefz[i];
                if (cx * cx + cy * cy + cz * cz > s.cl.cskin_half2) atomicOr(s.cl.rebuild, 1);
                const float4 pr = s.cl.pref[sl];
                const float px = ch.x - pr.x, py = ch.y - pr.y, pz = ch.z - pr.z;
                if (px * px + py * py + pz * pz > s.cl.pdisp2) atomicOr(s.cl.prune, 1);
            }
        }
        s.vx[i] = vx;
        s.vy[i] = vy;
        s.vz[i] = vz;
    }
    if (BOUNCE) {
        nprop = warp_sum_i(nprop);
        nacc = warp_sum_i(nacc);
        near = warp_sum_i(near);
        if (lane == 0) {
            if (nprop) atomicAdd(&cnt[0], (unsigned long long)nprop);
            if (nacc) atomicAdd(&cnt[1], (unsigned long long)nacc);
            if (near) atomicAdd(&cnt[2], (unsigned long long)near);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            if (cnt[0]) atomicAdd(&s.cnt[CNT_PROPOSALS], cnt[0]);
            if (cnt[1]) atomicAdd(&s.cnt[CNT_ACCEPTS], cnt[1]);
            if (cnt[2]) atomicAdd(&s.cnt[CNT_NEAR], cnt[2]);
        }
    }
}

// One jump half-step on the current velocities (component entry point).
__global__ void __launch_bounds__(NW * 32) k_jump_half(DevSys s, Params p, int cur, long long step, int stream_id,
                                                      int* Mout, int* Aout) {
    __shared__ JumpSmem js;
    __shared__ PropSmem ps;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int base = blockIdx.x * BOUNCE_GROUP;
    const int na = min(BOUNCE_GROUP, s.n - base);
    if (threadIdx.x == 0) {
        js.cnt[0] = js.cnt[1] = js.cnt[2] = 0ull;
    }
    for (int k = threadIdx.x; k < 129; k += blockDim.x) js.inv[k] = k ? __frcp_rn((float)k) : 0.f;
    if (warp == 0 && lane < na) {
        const int i = base + lane;
        jump_prep(s, p, js, lane, i, s.vx[i], s.vy[i], s.vz[i]);
    }
    __syncthreads();
    poisson_phase(s, p, js, base, na, step, (uint32_t)stream_id);
    jump_phase(s, p, js, ps, cur, base, na, step, (uint32_t)stream_id);
    if (warp == 0 && lane < na) {
        const int i = base + lane;
        s.vx[i] += (double)js.dv[lane][0];
        s.vy[i] += (double)js.dv[lane][1];
        s.vz[i] += (double)js.dv[lane][2];
        if (Mout) Mout[i] = js.M[lane];
        if (Aout) Aout[i] = js.nacc[lane];
    }
    if (threadIdx.x == 0) {
        atomicAdd(&s.cnt[CNT_PROPOSALS], js.cnt[0]);
        atomicAdd(&s.cnt[CNT_ACCEPTS], js.cnt[1]);
        atomicAdd(&s.cnt[CNT_NEAR], js.cnt[2]);
    }
}

__global__ void k_gradient(DevSys s, Params p, int part, int cur, double* out) {
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= s.n) return;
    int np;
    const float3 g = atom_gradient(s, p, cur, i, part, np);
    if (lane == 0) {
        out[3 * (size_t)i + 0] = g.x;
        out[3 * (size_t)i + 1] = g.y;
        out[3 * (size_t)i + 2] = g.z;
    }
}

// Pair sums of part `part` (atom_gradient) for every atom, one warp per
// atom, for the step kernel to read: a separate kernel with few registers
// keeps many more warps in flight on the partners' position gathers than the
// fused step kernel can.
__global__ void __launch_bounds__(256, 4) k_pairs(DevSys s, Params p, int step_off, int part) {
    chain_enter();
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (i >= s.n) return;
    const int cur = (int)((*s.step_base + step_off) & 1);
    int np = 0;
    const float3 g = atom_gradient(s, p, cur, i, part, np);
    if (lane == 0) s.g0[i] = make_float4(g.x, g.y, g.z, __int_as_float(np));
}

__global__ void k_advance(DevSys s, long long by) {
    chain_enter();
    *const_cast<long long*>(s.step_base) += by;
}

}  // namespace

// The pair sums a step boundary needs before its step kernel (their own
// kernel); returns whether the step kernel reads them (pre).
int launch_step_pairs(const DevSys& s, const Params& p, int integrator, int step_off, double hout, cudaStream_t st) {
    const int ext = integrator >= 3 ? 1 : 0;  // extended RESPA and RESPA1: bonded-only F_0
    int pre;
    if (s.cl.on) {
        // cluster pair sums (Newton's third law, fixed-point accumulators),
        // except at a boundary without pair sums (the extended splits between
        // outer kicks); F_0 takes the short-range list when there is one
        pre = (ext && hout == 0.0) ? 0 : 1;
        if (pre)
            launch_cluster_pairs(s, p, step_off, integrator != 0 ? 3 : 5, integrator != 0 && s.cl.nlists > 1 ? 1 : 0,
                                 st);
    } else {
        // all pairs (no cutoff): tiles, or the long candidate rows in their
        // own kernel; short rows (Coulomb on the jumps) stay in the step
        // kernel, and so does a boundary without pair sums (the extended
        // splits between outer kicks)
        const bool short_f0 = integrator != 0 && p.rshort2 < INFINITY;
        pre = ((ext && hout == 0.0) || short_f0) ? 0 : 1;
        if (pre && s.tl.on) launch_tile_pairs(s, p, step_off, integrator != 0 ? 3 : 5, st);
        else if (pre) launch_chained(k_pairs, (s.n + 7) / 8, 256, 0, st, s, p, step_off, integrator != 0 ? 3 : 5);
    }
    return pre;
}

void launch_step_kernel(const DevSys& s, const Params& p, int integrator, int variant, int step_off, double hr,
                        double hout, int pre, cudaStream_t st) {
    const int blocks = (s.n + BOUNCE_GROUP - 1) / BOUNCE_GROUP;
    const int ext = integrator >= 3 ? 1 : 0;
    // the thread-per-atom kernel where its preconditions hold: pair sums
    // from the cluster or tile kernel (or none at this boundary), and rare
    // proposals (s.lite, decided on the host from the jump bounds)
    if (s.lite && (s.cl.on || s.tl.on) && (pre || (ext && hout == 0.0))) {
        const int lb = (s.n + 255) / 256;
        if (integrator != 0) launch_chained(k_step_lite<1>, lb, 256, 0, st, s, p, variant, step_off, hr, ext, hout);
        else launch_chained(k_step_lite<0>, lb, 256, 0, st, s, p, variant, step_off, hr, 0, 0.0);
        return;
    }
    if (integrator != 0)
        launch_chained(k_step<1>, blocks, NW * 32, 0, st, s, p, variant, step_off, hr, ext, hout, pre);
    else launch_chained(k_step<0>, blocks, NW * 32, 0, st, s, p, variant, step_off, hr, 0, 0.0, pre);
}

void launch_step(const DevSys& s, const Params& p, int integrator, int variant, int step_off, double hr,
                 double hout, cudaStream_t st) {
    const int pre = launch_step_pairs(s, p, integrator, step_off, hout, st);
    launch_step_kernel(s, p, integrator, variant, step_off, hr, hout, pre, st);
}

void launch_jump_half(const DevSys& s, const Params& p, int cur, long long step, int stream_id, int* M, int* nacc,
                      cudaStream_t st) {
    const int blocks = (s.n + BOUNCE_GROUP - 1) / BOUNCE_GROUP;
    k_jump_half<<<blocks, NW * 32, 0, st>>>(s, p, cur, step, stream_id, M, nacc);
}

void launch_gradient(const DevSys& s, const Params& p, int part, int cur, double* out, cudaStream_t st) {
    const int wpb = 8;
    k_gradient<<<(s.n + wpb - 1) / wpb, wpb * 32, 0, st>>>(s, p, part, cur, out);
}

void launch_advance_step(const DevSys& s, long long by, cudaStream_t st) {
    launch_chained(k_advance, 1, 1, 0, st, s, by);
}
