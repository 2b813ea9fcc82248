// Differentiable direct-space pair forces for force matching (the pair
// terms of paper Sec. IV.A / V with trainable per-type parameters).
//
// Forward: F_i = -sum_j g(r_ij) d_ij, g = W'(r)/r, d_ij = q_i - q_j, over the
// candidate rows with r^2 < r_c^2, and E = sum_{i<j} W.  W = k q_a q_b / r
// (or k q_a q_b erfc(beta r)/r) + c12/r^12 - c6/r^6, c12 = 4 eps sigma^12,
// c6 = 4 eps sigma^6, with per-type charges q_t and symmetric sigma, eps.
// Backward for L(F, E) with upstream u_i = dL/dF_i and w = dL/dE:
//   dL/dq_i = sum_j [ -H(d_ij) (u_i - u_j) + w g d_ij ],
//             H(d) = g I + (g'(r)/r) d d^T (the pair Hessian of W);
//   dL/dtheta = sum_{i<j} [ -(dg/dtheta) (u_i - u_j).d_ij + w dW/dtheta ].
// One warp per atom, FP32 pair math; per-atom parameter partials in FP64,
// summed in a fixed order, so the gradients do not depend on scheduling.
#include "common.cuh"

namespace {

constexpr int MAXT = BOUNCE_MAXT;
constexpr int NPAR = MAXT + 2 * MAXT * MAXT;  // charges, sigma, eps (full tables)

struct DiffParams {
    float qt[MAXT];
    float sig[MAXT * MAXT];
    float eps[MAXT * MAXT];
    int T;
};

// Pair quantities for parameters p: g, dg/dr, W and the partial
// derivatives of g and W with respect to (q_product, c12, c6).
struct PairD {
    float g, gp, W;
    float dg_dqq, dW_dqq;   // per unit of k q_a q_b
    float dg_dc12, dg_dc6, dW_dc12, dW_dc6;
};

__device__ __forceinline__ PairD pair_terms_d(const Params& p, float r2, float qq, float c12, float c6) {
    PairD o;
    const float ir = rsqrt_nr(r2);
    const float r = r2 * ir;
    const float ir2 = ir * ir;
    float gc, gpc, wc;  // Coulomb g, g', W per unit qq
    if (p.ebeta > 0.f) {
        const float b = p.ebeta;
        const float ec = erfcf(b * r), ex = expf(-b * b * r2);
        const float c = p.e2b_sqrtpi;
        wc = ec * ir;
        const float dW = -(ec * ir2 + c * ex * ir);
        const float d2W = 2.f * ec * ir2 * ir + c * ex * (2.f * ir2 + 2.f * b * b);
        gc = dW * ir;
        gpc = d2W * ir - dW * ir2;
    } else {
        wc = ir;
        gc = -ir2 * ir;
        gpc = 3.f * ir2 * ir2;
    }
    const float ir6 = ir2 * ir2 * ir2;
    const float ir8 = ir6 * ir2;
    o.dg_dqq = gc;
    o.dW_dqq = wc;
    o.dg_dc12 = -12.f * ir6 * ir8;
    o.dg_dc6 = 6.f * ir8;
    o.dW_dc12 = ir6 * ir6;
    o.dW_dc6 = -ir6;
    o.g = qq * gc + c12 * o.dg_dc12 + c6 * o.dg_dc6;
    o.gp = qq * gpc + c12 * (168.f * ir8 * ir6 * ir) + c6 * (-48.f * ir8 * ir);
    o.W = qq * wc + c12 * o.dW_dc12 + c6 * o.dW_dc6;
    return o;
}

__device__ __forceinline__ void type_params(const DiffParams& dp, int ti, int tj, float& qq, float& c12, float& c6) {
    const float s = dp.sig[ti * MAXT + tj], e = dp.eps[ti * MAXT + tj];
    const float s2 = s * s, s6 = s2 * s2 * s2;
    qq = (float)KCOUL_D * dp.qt[ti] * dp.qt[tj];
    c12 = 4.f * e * s6 * s6;
    c6 = 4.f * e * s6;
}

__global__ void k_pair_fwd(DevSys s, Params p, DiffParams dp, int cur, double* F, double* eatom) {
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= s.n) return;
    const float4 hi = s.phi[cur][i], lo = s.plo[cur][i];
    const int ti = type_of(lo);
    const int n = s.nlong[i];
    const int* row = s.rows + (size_t)i * s.cap;
    float fx = 0.f, fy = 0.f, fz = 0.f, e = 0.f;
    for (int k = lane; k < n; k += 32) {
        const int j = row[k];
        const float4 hj = s.phi[cur][j], lj = s.plo[cur][j];
        const float3 d = pair_disp(p, hi, lo, hj, lj);
        const float r2 = d.x * d.x + d.y * d.y + d.z * d.z;
        if (!inside_cut(s, p, cur, i, j, r2)) continue;
        float qq, c12, c6;
        type_params(dp, ti, type_of(lj), qq, c12, c6);
        const PairD t = pair_terms_d(p, r2, qq, c12, c6);
        fx -= t.g * d.x;
        fy -= t.g * d.y;
        fz -= t.g * d.z;
        if (j > i) e += t.W;
    }
    fx = warp_sum_f(fx);
    fy = warp_sum_f(fy);
    fz = warp_sum_f(fz);
    e = warp_sum_f(e);
    if (lane == 0) {
        F[3 * (size_t)i] = fx;
        F[3 * (size_t)i + 1] = fy;
        F[3 * (size_t)i + 2] = fz;
        eatom[i] = e;
    }
}

// Backward: position gradient per atom and per-atom parameter partials
// (pairs j > i) into part[NPAR][n].
__global__ void k_pair_bwd(DevSys s, Params p, DiffParams dp, int cur, const double* U, double w, double* gpos,
                           double* part) {
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= s.n) return;
    const float4 hi = s.phi[cur][i], lo = s.plo[cur][i];
    const int ti = type_of(lo);
    const int n = s.nlong[i];
    const int* row = s.rows + (size_t)i * s.cap;
    const float uix = (float)U[3 * (size_t)i], uiy = (float)U[3 * (size_t)i + 1], uiz = (float)U[3 * (size_t)i + 2];
    const float wf = (float)w;
    float gx = 0.f, gy = 0.f, gz = 0.f;
    float pq[MAXT], ps[MAXT * MAXT], pe[MAXT * MAXT];
    for (int a = 0; a < MAXT; ++a) pq[a] = 0.f;
    for (int a = 0; a < MAXT * MAXT; ++a) ps[a] = pe[a] = 0.f;
    for (int k = lane; k < n; k += 32) {
        const int j = row[k];
        const float4 hj = s.phi[cur][j], lj = s.plo[cur][j];
        const float3 d = pair_disp(p, hi, lo, hj, lj);
        const float r2 = d.x * d.x + d.y * d.y + d.z * d.z;
        if (!inside_cut(s, p, cur, i, j, r2)) continue;
        const int tj = type_of(lj);
        float qq, c12, c6;
        type_params(dp, ti, tj, qq, c12, c6);
        const PairD t = pair_terms_d(p, r2, qq, c12, c6);
        const float dux = uix - (float)U[3 * (size_t)j], duy = uiy - (float)U[3 * (size_t)j + 1],
                    duz = uiz - (float)U[3 * (size_t)j + 2];
        const float r = sqrtf(r2);
        const float ddu = d.x * dux + d.y * duy + d.z * duz;
        const float h = t.gp / r * ddu;
        // -H (u_i - u_j) + w g d
        gx += -(t.g * dux + h * d.x) + wf * t.g * d.x;
        gy += -(t.g * duy + h * d.y) + wf * t.g * d.y;
        gz += -(t.g * duz + h * d.z) + wf * t.g * d.z;
        if (j > i) {
            // d/dtheta of -g (u_i - u_j).d + w W
            const float kq = (float)KCOUL_D;
            const float cq = -t.dg_dqq * ddu + wf * t.dW_dqq;  // per unit of k q_a q_b
            pq[ti] += cq * kq * dp.qt[tj];
            pq[tj] += cq * kq * dp.qt[ti];
            const float cc12 = -t.dg_dc12 * ddu + wf * t.dW_dc12;
            const float cc6 = -t.dg_dc6 * ddu + wf * t.dW_dc6;
            const float sg = dp.sig[ti * MAXT + tj], ep = dp.eps[ti * MAXT + tj];
            const float s2 = sg * sg, s5 = s2 * s2 * sg, s6 = s5 * sg, s11 = s6 * s5;
            const int a = min(ti, tj), b = max(ti, tj);
            ps[a * MAXT + b] += cc12 * 48.f * ep * s11 + cc6 * 24.f * ep * s5;
            pe[a * MAXT + b] += cc12 * 4.f * s6 * s6 + cc6 * 4.f * s6;
        }
    }
    gx = warp_sum_f(gx);
    gy = warp_sum_f(gy);
    gz = warp_sum_f(gz);
    if (lane == 0) {
        gpos[3 * (size_t)i] = gx;
        gpos[3 * (size_t)i + 1] = gy;
        gpos[3 * (size_t)i + 2] = gz;
    }
    for (int a = 0; a < MAXT; ++a) {
        const float v = warp_sum_f(pq[a]);
        if (lane == 0) part[(size_t)a * s.n + i] = v;
    }
    for (int a = 0; a < MAXT * MAXT; ++a) {
        const float v1 = warp_sum_f(ps[a]);
        const float v2 = warp_sum_f(pe[a]);
        if (lane == 0) {
            part[(size_t)(MAXT + a) * s.n + i] = v1;
            part[(size_t)(MAXT + MAXT * MAXT + a) * s.n + i] = v2;
        }
    }
}

// Fixed-order sums of `rows` per-atom arrays of length n: out[r] = sum_i x[r][i].
__global__ void k_rowsum(int n, int rows, const double* x, double* out) {
    __shared__ double red[256];
    for (int r = blockIdx.x; r < rows; r += gridDim.x) {
        double acc = 0.0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) acc += x[(size_t)r * n + i];
        red[threadIdx.x] = acc;
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
            if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[r] = red[0];
        __syncthreads();
    }
}

}  // namespace

int diff_param_count() { return NPAR; }

void launch_pair_forward(const DevSys& s, const Params& p, const float* qt, const float* sig, const float* eps, int T,
                         int cur, double* F, double* eatom, double* esum, cudaStream_t st) {
    DiffParams dp{};
    for (int a = 0; a < MAXT; ++a) dp.qt[a] = a < T ? qt[a] : 0.f;
    for (int a = 0; a < MAXT * MAXT; ++a) dp.sig[a] = sig[a], dp.eps[a] = eps[a];
    dp.T = T;
    const int wpb = 8;
    k_pair_fwd<<<(s.n + wpb - 1) / wpb, wpb * 32, 0, st>>>(s, p, dp, cur, F, eatom);
    k_rowsum<<<1, 256, 0, st>>>(s.n, 1, eatom, esum);
}

void launch_pair_backward(const DevSys& s, const Params& p, const float* qt, const float* sig, const float* eps, int T,
                          int cur, const double* U, double w, double* gpos, double* part, double* psum,
                          cudaStream_t st) {
    DiffParams dp{};
    for (int a = 0; a < MAXT; ++a) dp.qt[a] = a < T ? qt[a] : 0.f;
    for (int a = 0; a < MAXT * MAXT; ++a) dp.sig[a] = sig[a], dp.eps[a] = eps[a];
    dp.T = T;
    const int wpb = 8;
    k_pair_bwd<<<(s.n + wpb - 1) / wpb, wpb * 32, 0, st>>>(s, p, dp, cur, U, w, gpos, part);
    k_rowsum<<<NPAR, 256, 0, st>>>(s.n, NPAR, part, psum);
}
