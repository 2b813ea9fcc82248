// Fused per-step kernels of BOUNCE (B J A O A J B, paper Sec. III.C and the
// algorithm of Sec. IV.B) and BAOAB.
//
// Step fusion: B and J do not commute, but the end of step n (J then B/2)
// and the start of step n+1 (B/2 then J) act at the same positions.  So one
// launch per step does, for every atom, at positions q_n:
//     F_0(q_n)  ->  J(delta/2) [stream 2, step n-1]  ->  B(delta)
//               ->  J(delta/2) [stream 1, step n]   ->  A(delta/2) O A(delta/2)
// writing q_{n+1} to the other position buffer (J of atom i reads partners
// at q_n).  A run is a head launch (B/2 instead of J B), bodies, and a tail
// launch (J then B/2, no drift).
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

struct JumpSmem {
    double s[BOUNCE_GROUP];       // ||v|| (FP64)
    float sl[BOUNCE_GROUP];       // ||v|| L* (FP32)
    float vf[BOUNCE_GROUP][3];    // FP32 velocity at the start of the chain
    float dv[BOUNCE_GROUP][3];    // accumulated jump increment
    float muc[BOUNCE_GROUP];      // Poisson chunk mean (FP32)
    int nch[BOUNCE_GROUP];        // number of Poisson chunks
    int M[BOUNCE_GROUP];          // proposals of each atom (sum of its Poisson chunks)
    int nacc[BOUNCE_GROUP];
    int chp[BOUNCE_GROUP + 1];    // prefix of the chunk counts
    float inv[129];               // 1/k, k = 0..128 (round-to-nearest reciprocals)
    int next;
    unsigned long long cnt[3];    // proposals, accepts, near ties
};

// Lane-parallel (warp 0): quantities of the jump step of atom `a` that need FP64.
__device__ __forceinline__ void jump_prep(const DevSys& s, const Params& p, JumpSmem& js, int a, int i, double vx,
                                          double vy, double vz) {
    const double sp = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(vx, vx), __dmul_rn(vy, vy)), __dmul_rn(vz, vz)));
    const int t = s.type[i];
    const double Ls = p.Lstar_d[t];
    const int n = s.nlong[i];
    double mu = __dmul_rn(__dmul_rn(__dmul_rn(__dmul_rn(__dmul_rn(p.beta, sp), Ls), (double)n), p.dt), 0.5);
    if (!(mu <= 1e6)) {  // a blown-up state: report instead of drawing millions of proposals
        atomicOr(s.err, BERR_RATE);
        mu = 0.0;
    }
    int nch = 0;
    float muc = 0.f;
    if (mu > 0.0) {
        nch = (int)ceil(__ddiv_rn(mu, 16.0));
        muc = __double2float_rn(__ddiv_rn(mu, (double)nch));
    }
    js.s[a] = sp;
    js.sl[a] = __double2float_rn(__dmul_rn(sp, Ls));
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

// Poisson counts of the CTA's atoms (one half step): every thread takes
// whole chunks (chunk c of atom a inverts Poisson(mu_c) with the uniform of
// Philox slot 0x80000000 | c), one chunk per thread at a time, and adds its
// count to the atom's total.  Called by all threads of the CTA.
__device__ void poisson_phase(const DevSys& s, const Params& p, JumpSmem& js, int base, int na, long long step,
                              uint32_t stream) {
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int a = 0; a < na; ++a) {
            js.chp[a] = acc;
            acc += js.nch[a];
            js.M[a] = 0;
        }
        js.chp[na] = acc;
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
        // sequential search of the FP32 CDF (same operations as poisson_invert_f32)
        const float u = u24(x.x), mu_c = js.muc[lo];
        float pk = expneg_f32(mu_c), cdf = pk;
        int k = 0;
        while (u > cdf && k < 128) {
            ++k;
            const float q = __fmul_rn(__fmul_rn(pk, mu_c), js.inv[k]);
            const float cn = __fadd_rn(cdf, q);
            if (cn == cdf) break;
            pk = q;
            cdf = cn;
        }
        atomicAdd(&js.M[lo], k);
    }
    __syncthreads();
}

// Warp-cooperative jump chain of atom `a` (one half step).
__device__ void jump_chain(const DevSys& s, const Params& p, JumpSmem& js, int cur, int a, int i, long long step,
                           uint32_t stream) {
    const int lane = threadIdx.x & 31;
    const int M = js.M[a];
    float vx = js.vf[a][0], vy = js.vf[a][1], vz = js.vf[a][2];
    float dvx = 0.f, dvy = 0.f, dvz = 0.f;
    int nacc = 0, near = 0;
    if (M > 0) {
        const float4 hi = s.phi[cur][i], lo = s.plo[cur][i];
        const float qi = hi.w;
        const int ti = type_of(lo);
        const int n = s.nlong[i];
        const int* row = s.rows + (size_t)i * s.cap;
        const float sl = js.sl[a];
        const double sp = js.s[a], Ls = p.Lstar_d[ti];
        for (int kb = 0; kb < M; kb += 32) {
            const int k = kb + lane + 1;
            const bool act = k <= M;
            float gx = 0.f, gy = 0.f, gz = 0.f, uf = 1.f;
            uint32_t x1 = 0, x2 = 0;
            if (act) {
                const uint4 x = rng_atom(s, p, (uint32_t)k, i, step, stream);
                const int J = (int)__umulhi(x.x, (uint32_t)n);
                const int j = row[J];
                const float4 hj = s.phi[cur][j], lj = s.plo[cur][j];
                const float3 d = pair_disp(p, hi, lo, hj, lj);
                const float r2 = d.x * d.x + d.y * d.y + d.z * d.z;
                if (inside_cut(s, p, cur, i, j, r2)) {
                    const float r = sqrtf(r2);
                    const float w = chi_of(p, r) * pair_dW_over_r(p, r2, p.kcoul * qi * hj.w, ti * BOUNCE_MAXT + type_of(lj));
                    gx = w * d.x;
                    gy = w * d.y;
                    gz = w * d.z;
                }
                uf = u24(x.y);
                x1 = x.y;
                x2 = x.z;
            }
            int start = 0;
            while (true) {
                // decide with the current velocity: accept iff U ||v|| L* < v . F
                const float af = vx * gx + vy * gy + vz * gz;
                const float thr = uf * sl;
                const float err = 4e-6f * (thr + fabsf(vx * gx) + fabsf(vy * gy) + fabsf(vz * gz)) + 2.4e-7f * sl;
                int dec = (thr + err < af) ? 1 : ((thr - err > af) ? 0 : 2);
                const bool live = act && lane >= start;
                if (__any_sync(0xffffffffu, live && dec == 2)) {
                    if (live && dec == 2) dec = exact_decision(vx, vy, vz, gx, gy, gz, x1, x2, sp, Ls);
                }
                const uint32_t acc = __ballot_sync(0xffffffffu, live && dec == 1);
                const int f = acc ? __ffs(acc) - 1 : 32;
                // near ties among the decisions that stand (lanes start..f)
                const bool stands = live && lane <= f;
                if (stands && fabsf(thr - af) < 1e-6f * sl) ++near;
                if (!acc) break;
                const float fx = __shfl_sync(0xffffffffu, gx, f), fy = __shfl_sync(0xffffffffu, gy, f),
                            fz = __shfl_sync(0xffffffffu, gz, f);
                const float aa = vx * fx + vy * fy + vz * fz;
                const float ff = fx * fx + fy * fy + fz * fz;
                const float coef = (aa + aa) / ff;
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
    }
    near = warp_sum_i(near);
    if (lane == 0) {
        js.dv[a][0] = dvx;
        js.dv[a][1] = dvy;
        js.dv[a][2] = dvz;
        js.nacc[a] = nacc;
        atomicAdd(&js.cnt[0], (unsigned long long)M);
        atomicAdd(&js.cnt[1], (unsigned long long)nacc);
        atomicAdd(&js.cnt[2], (unsigned long long)near);
    }
}

// Warp-cooperative gradient of atom i: part 0 = full (long rows, chi = 1),
// 1 = short (short rows, 1 - chi), 2 = long (long rows, chi), 3 = short
// pairs without bonded terms, 4 = bonded terms only; bonded terms are added
// for parts 0, 1 and 4.
__device__ float3 atom_gradient(const DevSys& s, const Params& p, int cur, int i, int part, int& npairs) {
    const int lane = threadIdx.x & 31;
    const float4 hi = s.phi[cur][i], lo = s.plo[cur][i];
    const float qi = hi.w;
    const int ti = type_of(lo);
    const bool shortrows = part == 1 || part == 3;
    const int n = part == 4 ? 0 : (shortrows ? s.nshort[i] : s.nlong[i]);
    const int* row = shortrows ? s.srows + (size_t)i * s.caps : s.rows + (size_t)i * s.cap;
    float gx = 0.f, gy = 0.f, gz = 0.f;
    for (int k = lane; k < n; k += 32) {
        const int j = row[k];
        const float4 hj = s.phi[cur][j], lj = s.plo[cur][j];
        const float3 d = pair_disp(p, hi, lo, hj, lj);
        const float r2 = d.x * d.x + d.y * d.y + d.z * d.z;
        if (inside_cut(s, p, cur, i, j, r2)) {
            float w = pair_dW_over_r(p, r2, p.kcoul * qi * hj.w, ti * BOUNCE_MAXT + type_of(lj));
            if (part != 0) {
                const float c = chi_of(p, sqrtf(r2));
                w *= part == 2 ? c : 1.f - c;
            }
            gx += w * d.x;
            gy += w * d.y;
            gz += w * d.z;
        }
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
__global__ void __launch_bounds__(NW * 32, 4) k_step(DevSys s, Params p, int variant, int step_off, double hr,
                                                     int ext, double hout) {
    __shared__ float sG[BOUNCE_GROUP][3];
    __shared__ float sGp[BOUNCE_GROUP][3];
    __shared__ double sV[BOUNCE_GROUP][3];
    __shared__ JumpSmem js;
    __shared__ unsigned long long sPairs;
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
    __syncthreads();
    // F_0 (BOUNCE) or the full gradient (BAOAB) at q_n
    for (int a = warp; a < na; a += NW) {
        int np = 0, np2 = 0;
        const float3 g = atom_gradient(s, p, cur, base + a, ext ? 4 : (BOUNCE ? 1 : 0), np);
        float3 gp = make_float3(0.f, 0.f, 0.f);
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
    if (warp == 0 && lane < na) {
        const int i = base + lane;
        const double vx = s.vx[i], vy = s.vy[i], vz = s.vz[i];
        sV[lane][0] = vx;
        sV[lane][1] = vy;
        sV[lane][2] = vz;
        if (do_j2) jump_prep(s, p, js, lane, i, vx, vy, vz);
    }
    if (threadIdx.x == 0) js.next = 0;
    __syncthreads();
    if (do_j2) {
        poisson_phase(s, p, js, base, na, step - 1, BOUNCE_STREAM_J2);
        for (;;) {
            int a = 0;
            if (lane == 0) a = atomicAdd(&js.next, 1);
            a = __shfl_sync(0xffffffffu, a, 0);
            if (a >= na) break;
            jump_chain(s, p, js, cur, a, base + a, step - 1, BOUNCE_STREAM_J2);
        }
        __syncthreads();
    }
    if (warp == 0 && lane < na) {
        const int i = base + lane;
        double vx = sV[lane][0], vy = sV[lane][1], vz = sV[lane][2];
        if (do_j2) {
            vx += (double)js.dv[lane][0];
            vy += (double)js.dv[lane][1];
            vz += (double)js.dv[lane][2];
        }
        const double c = hk * s.kick[i];
        vx -= c * (double)sG[lane][0];
        vy -= c * (double)sG[lane][1];
        vz -= c * (double)sG[lane][2];
        if (hr != 0.0) {
            const double cr = hr * s.kick[i];
            vx -= cr * s.grecip[i];
            vy -= cr * s.grecip[s.n + i];
            vz -= cr * s.grecip[2 * (size_t)s.n + i];
        }
        if (ext && hout != 0.0) {
            const double co = hout * s.kick[i];
            vx -= co * (double)sGp[lane][0];
            vy -= co * (double)sGp[lane][1];
            vz -= co * (double)sGp[lane][2];
        }
        sV[lane][0] = vx;
        sV[lane][1] = vy;
        sV[lane][2] = vz;
        if (do_j1) jump_prep(s, p, js, lane, i, vx, vy, vz);
    }
    if (threadIdx.x == 0) js.next = 0;
    __syncthreads();
    if (do_j1) {
        poisson_phase(s, p, js, base, na, step, BOUNCE_STREAM_J1);
        for (;;) {
            int a = 0;
            if (lane == 0) a = atomicAdd(&js.next, 1);
            a = __shfl_sync(0xffffffffu, a, 0);
            if (a >= na) break;
            jump_chain(s, p, js, cur, a, base + a, step, BOUNCE_STREAM_J1);
        }
        __syncthreads();
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
            double x = s.qx[cur][i] + h * vx, y = s.qy[cur][i] + h * vy, z = s.qz[cur][i] + h * vz;
            // O: Box-Muller on Philox slot 0, stream 0
            const uint4 r = rng_atom(s, p, 0u, i, step, BOUNCE_STREAM_O);
            const float ra = sqrtf(-2.f * logf(u24_open0(r.x)));
            float sn, cs;
            sincospif(2.f * u24(r.y), &sn, &cs);
            const float g2 = sqrtf(-2.f * logf(u24_open0(r.z))) * cospif(2.f * u24(r.w));
            const double sd = s.osd[i];
            vx = p.c1 * vx + sd * (double)(ra * cs);
            vy = p.c1 * vy + sd * (double)(ra * sn);
            vz = p.c1 * vz + sd * (double)g2;
            x += h * vx;
            y += h * vy;
            z += h * vz;
            s.qx[nxt][i] = x;
            s.qy[nxt][i] = y;
            s.qz[nxt][i] = z;
            double wx = x, wy = y, wz = z;
            if (p.periodic) {
                wx -= p.Ld[0] * floor(x / p.Ld[0]);
                wy -= p.Ld[1] * floor(y / p.Ld[1]);
                wz -= p.Ld[2] * floor(z / p.Ld[2]);
            }
            const float hx = __double2float_rn(wx), hy = __double2float_rn(wy), hz = __double2float_rn(wz);
            const float4 oldh = s.phi[cur][i], oldl = s.plo[cur][i];
            s.phi[nxt][i] = make_float4(hx, hy, hz, oldh.w);
            s.plo[nxt][i] = make_float4(__double2float_rn(wx - (double)hx), __double2float_rn(wy - (double)hy),
                                        __double2float_rn(wz - (double)hz), oldl.w);
            const double ex = x - s.refx[i], ey = y - s.refy[i], ez = z - s.refz[i];
            if (ex * ex + ey * ey + ez * ez > p.skin_half2) atomicOr(s.rebuild, 1);
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

// One jump half-step on the current velocities (component entry point).
__global__ void __launch_bounds__(NW * 32) k_jump_half(DevSys s, Params p, int cur, long long step, int stream_id,
                                                      int* Mout, int* Aout) {
    __shared__ JumpSmem js;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int base = blockIdx.x * BOUNCE_GROUP;
    const int na = min(BOUNCE_GROUP, s.n - base);
    if (threadIdx.x == 0) {
        js.cnt[0] = js.cnt[1] = js.cnt[2] = 0ull;
        js.next = 0;
    }
    for (int k = threadIdx.x; k < 129; k += blockDim.x) js.inv[k] = k ? __frcp_rn((float)k) : 0.f;
    if (warp == 0 && lane < na) {
        const int i = base + lane;
        jump_prep(s, p, js, lane, i, s.vx[i], s.vy[i], s.vz[i]);
    }
    __syncthreads();
    poisson_phase(s, p, js, base, na, step, (uint32_t)stream_id);
    for (;;) {
        int a = 0;
        if (lane == 0) a = atomicAdd(&js.next, 1);
        a = __shfl_sync(0xffffffffu, a, 0);
        if (a >= na) break;
        jump_chain(s, p, js, cur, a, base + a, step, (uint32_t)stream_id);
    }
    __syncthreads();
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

__global__ void k_advance(DevSys s, long long by) { *const_cast<long long*>(s.step_base) += by; }

}  // namespace

void launch_step(const DevSys& s, const Params& p, int integrator, int variant, int step_off, double hr,
                 double hout, cudaStream_t st) {
    const int blocks = (s.n + BOUNCE_GROUP - 1) / BOUNCE_GROUP;
    const int ext = integrator == 3 ? 1 : 0;
    if (integrator != 0) k_step<1><<<blocks, NW * 32, 0, st>>>(s, p, variant, step_off, hr, ext, hout);
    else k_step<0><<<blocks, NW * 32, 0, st>>>(s, p, variant, step_off, hr, 0, 0.0);
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

void launch_advance_step(const DevSys& s, long long by, cudaStream_t st) { k_advance<<<1, 1, 0, st>>>(s, by); }
