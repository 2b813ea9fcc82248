// Energies of the current state (unsplit W, paper Sec. IV.A / V) and the
// position packing used after a state upload.
//
// Pair energies: one warp per atom sums W over the members j > i of its row
// with r < r_c (FP32 per pair, FP32 per lane, FP64 across lanes); bonded and
// kinetic terms per atom in FP64.  The per-atom terms are then summed by one
// CTA in a fixed order, so totals are deterministic.
#include "common.cuh"

namespace {

// terms layout: [5][n] = coulomb, lj, bond, angle, kinetic per atom
__global__ void k_atom_energies(DevSys s, Params p, int cur, double* terms) {
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= s.n) return;
    const float4 hi = s.phi[cur][i], lo = s.plo[cur][i];
    const int ti = type_of(lo);
    const int n = s.nlong[i];
    const int* row = s.rows + (size_t)i * s.cap;
    float ec = 0.f, el = 0.f;
    for (int k = lane; k < n; k += 32) {
        const int j = row[k];
        if (j <= i) continue;
        const float4 hj = s.phi[cur][j], lj = s.plo[cur][j];
        const float3 d = pair_disp(p, hi, lo, hj, lj);
        const float r2 = d.x * d.x + d.y * d.y + d.z * d.z;
        if (inside_cut(s, p, cur, i, j, r2)) {
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
    // bonded terms owned by atom i: bonds with i < partner, angles at their vertex
    double eb = 0.0, ea = 0.0;
    for (int t = s.bt_off[i] + lane; t < s.bt_off[i + 1]; t += 32) {
        const int4 b = s.bt_idx[t];
        const float2 kp = s.bt_par[t];
        if (b.x == 0 && i < b.y) {
            const float3 d = pair_disp(p, hi, lo, s.phi[cur][b.y], s.plo[cur][b.y]);
            const float r = sqrtf(d.x * d.x + d.y * d.y + d.z * d.z);
            eb += (double)(kp.x * (r - kp.y) * (r - kp.y));
        } else if (b.x == 2) {
            const float4 ha = s.phi[cur][b.y], la = s.plo[cur][b.y], hc = s.phi[cur][b.z], lc = s.plo[cur][b.z];
            const float3 u = pair_disp(p, ha, la, hi, lo);
            const float3 w = pair_disp(p, hc, lc, hi, lo);
            float cs = (u.x * w.x + u.y * w.y + u.z * w.z) *
                       rsqrt_nr((u.x * u.x + u.y * u.y + u.z * u.z) * (w.x * w.x + w.y * w.y + w.z * w.z));
            cs = fminf(fmaxf(cs, -1.f), 1.f);
            const float th = acosf(cs) - kp.y;
            ea += (double)(kp.x * th * th);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        eb += __shfl_xor_sync(0xffffffffu, eb, o);
        ea += __shfl_xor_sync(0xffffffffu, ea, o);
    }
    if (lane == 0) {
        const double vx = s.vx[i], vy = s.vy[i], vz = s.vz[i];
        terms[0 * (size_t)s.n + i] = dc;
        terms[1 * (size_t)s.n + i] = dl;
        terms[2 * (size_t)s.n + i] = eb;
        terms[3 * (size_t)s.n + i] = ea;
        // 1/2 m v^2 with m = 4.184e-4 / kick, in kcal/mol: 1/2 v^2 / kick
        terms[4 * (size_t)s.n + i] = 0.5 * (vx * vx + vy * vy + vz * vz) / s.kick[i];
    }
}

// Fixed-order sum of T per-atom term arrays: each of the first-pass CTAs
// sums a fixed slice of every array, then one CTA adds the per-CTA partials
// in CTA order, so totals do not depend on scheduling.
constexpr int SUM_CTAS = 128;

template <int T>
__global__ void k_sum_pass1(int n, const double* terms, double* partial) {
    __shared__ double part[T][256];
    const int per = (n + SUM_CTAS - 1) / SUM_CTAS;
    const int b = blockIdx.x * per, e = min(n, b + per);
    for (int t = 0; t < T; ++t) {
        double acc = 0.0;
        for (int i = b + threadIdx.x; i < e; i += blockDim.x) acc += terms[(size_t)t * n + i];
        part[t][threadIdx.x] = acc;
    }
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int t = 0; t < T; ++t) part[t][threadIdx.x] += part[t][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < T) partial[threadIdx.x * SUM_CTAS + blockIdx.x] = part[threadIdx.x][0];
}

template <int T>
__global__ void k_sum_pass2(const double* partial, double* out) {
    __shared__ double part[T][SUM_CTAS];
    for (int t = 0; t < T; ++t) part[t][threadIdx.x] = partial[t * SUM_CTAS + threadIdx.x];
    __syncthreads();
    for (int w = SUM_CTAS / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int t = 0; t < T; ++t) part[t][threadIdx.x] += part[t][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < T) out[threadIdx.x] = part[threadIdx.x][0];
}

// Split FP32 copies (hi + lo) of the FP64 positions of buffer `cur`;
// positions are wrapped into the box for periodic systems.
__global__ void k_pack(DevSys s, Params p, int cur) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < s.n; i += gridDim.x * blockDim.x) {
        double x = s.qx[cur][i], y = s.qy[cur][i], z = s.qz[cur][i];
        if (p.periodic) {
            x = wrap_box(x, p.Ld[0], p.iLd[0]);
            y = wrap_box(y, p.Ld[1], p.iLd[1]);
            z = wrap_box(z, p.Ld[2], p.iLd[2]);
        }
        const float hx = __double2float_rn(x), hy = __double2float_rn(y), hz = __double2float_rn(z);
        const float4 oh = s.phi[cur][i];
        const float4 ol = s.plo[cur][i];
        s.phi[cur][i] = make_float4(hx, hy, hz, oh.w);
        s.plo[cur][i] = make_float4(__double2float_rn(x - (double)hx), __double2float_rn(y - (double)hy),
                                    __double2float_rn(z - (double)hz), ol.w);
    }
}

}  // namespace

void launch_energies(const DevSys& s, const Params& p, int cur, double* terms, cudaStream_t st) {
    const int wpb = 8;
    k_atom_energies<<<(s.n + wpb - 1) / wpb, wpb * 32, 0, st>>>(s, p, cur, terms);
    // terms holds 6 n doubles: 5 n per-atom terms, then 5 * SUM_CTAS partials (n >= 640) or
    // fewer atoms: the partials go after the totals slot in any case
    double* partial = terms + 5 * (size_t)s.n + 8;
    k_sum_pass1<5><<<SUM_CTAS, 256, 0, st>>>(s.n, terms, partial);
    k_sum_pass2<5><<<1, SUM_CTAS, 0, st>>>(partial, terms + 5 * (size_t)s.n);
}

// State in: interleaved q[n][3], v[n][3] (device) -> FP64 SoA at buffer cur.
__global__ void k_state_in(DevSys s, const double* q, const double* v, int cur) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < s.n; i += gridDim.x * blockDim.x) {
        s.qx[cur][i] = q[3 * (size_t)i];
        s.qy[cur][i] = q[3 * (size_t)i + 1];
        s.qz[cur][i] = q[3 * (size_t)i + 2];
        s.vx[i] = v[3 * (size_t)i];
        s.vy[i] = v[3 * (size_t)i + 1];
        s.vz[i] = v[3 * (size_t)i + 2];
    }
}

// State out: FP64 SoA of the current step (read on the device) -> interleaved
// q[n][3], v[n][3] (device; either may be null).
__global__ void k_state_out(DevSys s, double* q, double* v) {
    const int cur = (int)(*s.step_base & 1);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < s.n; i += gridDim.x * blockDim.x) {
        if (q) {
            q[3 * (size_t)i] = s.qx[cur][i];
            q[3 * (size_t)i + 1] = s.qy[cur][i];
            q[3 * (size_t)i + 2] = s.qz[cur][i];
        }
        if (v) {
            v[3 * (size_t)i] = s.vx[i];
            v[3 * (size_t)i + 1] = s.vy[i];
            v[3 * (size_t)i + 2] = s.vz[i];
        }
    }
}

void launch_state_in(const DevSys& s, const double* q, const double* v, int cur, cudaStream_t st) {
    k_state_in<<<(s.n + 255) / 256, 256, 0, st>>>(s, q, v, cur);
}

void launch_state_out(const DevSys& s, double* q, double* v, cudaStream_t st) {
    k_state_out<<<(s.n + 255) / 256, 256, 0, st>>>(s, q, v);
}

void launch_pack_positions(const DevSys& s, const Params& p, int cur, cudaStream_t st) {
    k_pack<<<(s.n + 255) / 256, 256, 0, st>>>(s, p, cur);
}
