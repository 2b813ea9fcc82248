// Reciprocal-space Ewald by smooth particle-mesh Ewald (Essmann et al.,
// J. Chem. Phys. 103, 8577 (1995)) for periodic boxes; paper Sec. V puts
// grad E_recip in F_0 (basic BOUNCE) or on the RESPA outer step.
//
// Pipeline (all on the device, one launch each):
//   spread    per atom, order-n cardinal B-spline weights from the FP64
//             fractional coordinates; charge * weights added to an int64
//             fixed-point grid (2^40 scale), so the grid is bit-identical
//             whatever the atomic order;
//   load      fixed point -> FP32 complex grid; clears the int64 grid;
//   dft x3    forward transform, one CTA per grid line: the line and a
//             twiddle table sit in shared memory and each output is a direct
//             sum over the line (K^2 work per line, FP32);
//   convolve  multiply by the influence function B(m) C(m) (FP32 table made
//             on the host in FP64) and accumulate the energy partials
//             sum B C |F(Q)|^2 per CTA (FP64);
//   dft x3    inverse transform (no 1/K normalisation);
//   gather    per atom, q K/L sum dM M M conv (FP32) plus the removal of the
//             same-molecule pairs, -k q_i q_j erf(beta r)/r, into an FP64
//             gradient (SoA) that the step kernel kicks with.
#include <algorithm>

#include "common.cuh"

namespace {

constexpr double FIX = 1099511627776.0;  // 2^40
constexpr int MAX_ORDER = 8;

// M_n(fr + t), t = 0..n-1, and dM_n/dx at the same points, by the recursion
// M_{k+1}(x) = (x M_k(x) + (k + 1 - x) M_k(x - 1)) / k from M_2.
__device__ __forceinline__ void bspline_weights(float fr, int n, float* w, float* dw) {
    float a[MAX_ORDER + 1];
    for (int t = 0; t <= n; ++t) a[t] = 0.f;
    a[0] = fr;
    a[1] = 1.f - fr;
    for (int k = 2; k < n; ++k) {
        if (k == n - 1) {
            // derivative from M_{n-1}: M_n'(fr + t) = M_{n-1}(fr + t) - M_{n-1}(fr + t - 1)
            for (int t = 0; t < n; ++t) dw[t] = a[t] - (t > 0 ? a[t - 1] : 0.f);
        }
        for (int t = k; t >= 0; --t) {
            const float x = fr + (float)t;
            a[t] = (x * a[t] + ((float)(k + 1) - x) * (t > 0 ? a[t - 1] : 0.f)) / (float)k;
        }
    }
    if (n == 2) {
        dw[0] = 1.f;
        dw[1] = -1.f;
    }
    for (int t = 0; t < n; ++t) w[t] = a[t];
}

__device__ __forceinline__ void frac_coord(double x, double L, int K, int& fl, float& fr) {
    const double f = __ddiv_rn(x, L);
    const double u = (f - floor(f)) * (double)K;
    double g = floor(u);
    fl = (int)g;
    fr = (float)(u - g);
    if (fl >= K) fl -= K;
}

__global__ void k_pme_spread(DevSys s, DevPme m, int step_off) {
    const int cur = (int)((*s.step_base + step_off) & 1);
    const int n = m.order;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < s.n; i += gridDim.x * blockDim.x) {
        int f[3];
        float fr[3];
        frac_coord(s.qx[cur][i], m.L[0], m.K[0], f[0], fr[0]);
        frac_coord(s.qy[cur][i], m.L[1], m.K[1], f[1], fr[1]);
        frac_coord(s.qz[cur][i], m.L[2], m.K[2], f[2], fr[2]);
        float w[3][MAX_ORDER], dw[3][MAX_ORDER];
        for (int d = 0; d < 3; ++d) bspline_weights(fr[d], n, w[d], dw[d]);
        const float q = s.phi[cur][i].w;
        for (int a = 0; a < n; ++a) {
            const int ix = (f[0] - a + m.K[0]) % m.K[0];
            const float qa = q * w[0][a];
            for (int b = 0; b < n; ++b) {
                const int iy = (f[1] - b + m.K[1]) % m.K[1];
                const float qab = qa * w[1][b];
                const size_t row = ((size_t)ix * m.K[1] + iy) * m.K[2];
                for (int c = 0; c < n; ++c) {
                    const int iz = (f[2] - c + m.K[2]) % m.K[2];
                    const long long v = __double2ll_rn((double)(qab * w[2][c]) * FIX);
                    atomicAdd(&m.qgrid[row + iz], (unsigned long long)v);
                }
            }
        }
    }
}

__global__ void k_pme_load(DevPme m) {
    const size_t N = (size_t)m.K[0] * m.K[1] * m.K[2];
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < N; k += (size_t)gridDim.x * blockDim.x) {
        const long long v = (long long)m.qgrid[k];
        m.cgrid[k] = make_float2((float)((double)v / FIX), 0.f);
        m.qgrid[k] = 0ull;
    }
}

// Direct DFT of every line along `axis` (0 = x, 1 = y, 2 = z) of the
// K0 x K1 x K2 grid (z fastest): X_k = sum_j x_j exp(sign 2 pi i j k / K).
__global__ void k_pme_dft(DevPme m, int axis, float sign) {
    extern __shared__ float2 sh[];
    const int K = m.K[axis];
    float2* line = sh;
    float2* tw = sh + K;
    const int l = blockIdx.x;
    size_t base, stride;
    if (axis == 2) {
        base = (size_t)l * m.K[2];
        stride = 1;
    } else if (axis == 1) {
        const int kx = l / m.K[2], kz = l % m.K[2];
        base = (size_t)kx * m.K[1] * m.K[2] + kz;
        stride = m.K[2];
    } else {
        base = (size_t)l;  // l = ky * K2 + kz
        stride = (size_t)m.K[1] * m.K[2];
    }
    for (int j = threadIdx.x; j < K; j += blockDim.x) {
        line[j] = m.cgrid[base + j * stride];
        float sn, cs;
        sincospif(2.f * (float)j / (float)K, &sn, &cs);
        tw[j] = make_float2(cs, sign * sn);
    }
    __syncthreads();
    float2 out[4];
    int cnt = 0;
    for (int k = threadIdx.x; k < K; k += blockDim.x, ++cnt) {
        float re = 0.f, im = 0.f;
        int idx = 0;
        for (int j = 0; j < K; ++j) {
            const float2 x = line[j], t = tw[idx];
            re = fmaf(x.x, t.x, fmaf(-x.y, t.y, re));
            im = fmaf(x.x, t.y, fmaf(x.y, t.x, im));
            idx += k;
            if (idx >= K) idx -= K;
        }
        out[cnt] = make_float2(re, im);
    }
    __syncthreads();
    cnt = 0;
    for (int k = threadIdx.x; k < K; k += blockDim.x, ++cnt) m.cgrid[base + k * stride] = out[cnt];
}

// F(Q) <- B C F(Q); energy partial sum B C |F(Q)|^2 of this CTA into eterm.
__global__ void k_pme_convolve(DevPme m) {
    __shared__ double red[256];
    const size_t N = (size_t)m.K[0] * m.K[1] * m.K[2];
    double e = 0.0;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < N; k += (size_t)gridDim.x * blockDim.x) {
        const float2 c = m.cgrid[k];
        const float b = m.bc[k];
        e += (double)b * ((double)c.x * c.x + (double)c.y * c.y);
        m.cgrid[k] = make_float2(b * c.x, b * c.y);
    }
    red[threadIdx.x] = e;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) m.eterm[blockIdx.x] = red[0];
}

// Gradient of E_recip + E_excl per atom (FP64 SoA), and the exclusion energy
// of the pairs (i, j > i) owned by atom i (for bounce_get_energies).
__global__ void k_pme_gather(DevSys s, Params p, DevPme m, int step_off) {
    const int cur = (int)((*s.step_base + step_off) & 1);
    const int n = m.order;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < s.n; i += gridDim.x * blockDim.x) {
        int f[3];
        float fr[3];
        frac_coord(s.qx[cur][i], m.L[0], m.K[0], f[0], fr[0]);
        frac_coord(s.qy[cur][i], m.L[1], m.K[1], f[1], fr[1]);
        frac_coord(s.qz[cur][i], m.L[2], m.K[2], f[2], fr[2]);
        float w[3][MAX_ORDER], dw[3][MAX_ORDER];
        for (int d = 0; d < 3; ++d) bspline_weights(fr[d], n, w[d], dw[d]);
        float gx = 0.f, gy = 0.f, gz = 0.f;
        for (int a = 0; a < n; ++a) {
            const int ix = (f[0] - a + m.K[0]) % m.K[0];
            for (int b = 0; b < n; ++b) {
                const int iy = (f[1] - b + m.K[1]) % m.K[1];
                const size_t row = ((size_t)ix * m.K[1] + iy) * m.K[2];
                float sx = 0.f, sy = 0.f, sz = 0.f;
                for (int c = 0; c < n; ++c) {
                    const int iz = (f[2] - c + m.K[2]) % m.K[2];
                    const float cv = m.cgrid[row + iz].x;
                    sx += cv * w[2][c];
                    sz += cv * dw[2][c];
                }
                gx += dw[0][a] * w[1][b] * sx;
                gy += w[0][a] * dw[1][b] * sx;
                gz += w[0][a] * w[1][b] * sz;
                (void)sy;
            }
        }
        const float4 hi = s.phi[cur][i], lo = s.plo[cur][i];
        const double kq = KCOUL_D * (double)hi.w;
        double Gx = kq * (double)gx * (m.K[0] / m.L[0]);
        double Gy = kq * (double)gy * (m.K[1] / m.L[1]);
        double Gz = kq * (double)gz * (m.K[2] / m.L[2]);
        // same-molecule pairs: -k q_i q_j erf(beta r)/r
        double ex = 0.0;
        for (int t = m.ex_off[i]; t < m.ex_off[i + 1]; ++t) {
            const int j = m.ex_idx[t];
            const float4 hj = s.phi[cur][j], lj = s.plo[cur][j];
            const float3 d = pair_disp(p, hi, lo, hj, lj);
            const float r2 = d.x * d.x + d.y * d.y + d.z * d.z;
            const float r = sqrtf(r2);
            const float br = m.beta * r;
            const float qq = (float)KCOUL_D * hi.w * hj.w;
            const float e = erff(br) / r;
            // d/dr (erf(b r)/r) = 2b/sqrt(pi) exp(-b^2 r^2)/r - erf(b r)/r^2
            const float dwr = -qq * (m.two_b_sqrtpi * expf(-br * br) / r - e / r) / r;
            Gx += (double)(dwr * d.x);
            Gy += (double)(dwr * d.y);
            Gz += (double)(dwr * d.z);
            if (j > i) ex += -(double)qq * (double)e;
        }
        m.grad[i] = Gx;
        m.grad[s.n + i] = Gy;
        m.grad[2 * (size_t)s.n + i] = Gz;
        m.eexcl[i] = ex;
    }
}

__global__ void k_pme_energy_sum(DevPme m, int nparts, int n, double* out) {
    __shared__ double red[2][256];
    double a = 0.0, b = 0.0;
    for (int k = threadIdx.x; k < nparts; k += blockDim.x) a += m.eterm[k];
    for (int k = threadIdx.x; k < n; k += blockDim.x) b += m.eexcl[k];
    red[0][threadIdx.x] = a;
    red[1][threadIdx.x] = b;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            red[0][threadIdx.x] += red[0][threadIdx.x + w];
            red[1][threadIdx.x] += red[1][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = 0.5 * KCOUL_D * red[0][0];  // E_recip
        out[1] = red[1][0];                    // E_excl
    }
}

}  // namespace

constexpr int PME_CONV_CTAS = 256;

void launch_pme(const DevSys& s, const Params& p, const DevPme& m, int step_off, cudaStream_t st) {
    const int tb = 128;
    k_pme_spread<<<(s.n + tb - 1) / tb, tb, 0, st>>>(s, m, step_off);
    const size_t N = (size_t)m.K[0] * m.K[1] * m.K[2];
    k_pme_load<<<(int)std::min<size_t>((N + 255) / 256, 4096), 256, 0, st>>>(m);
    const int lines[3] = {m.K[1] * m.K[2], m.K[0] * m.K[2], m.K[0] * m.K[1]};
    for (int axis = 2; axis >= 0; --axis)
        k_pme_dft<<<lines[axis], 128, 2 * m.K[axis] * sizeof(float2), st>>>(m, axis, -1.f);
    k_pme_convolve<<<PME_CONV_CTAS, 256, 0, st>>>(m);
    for (int axis = 2; axis >= 0; --axis)
        k_pme_dft<<<lines[axis], 128, 2 * m.K[axis] * sizeof(float2), st>>>(m, axis, 1.f);
    k_pme_gather<<<(s.n + tb - 1) / tb, tb, 0, st>>>(s, p, m, step_off);
}

void launch_pme_energy(const DevPme& m, int n, double* out, cudaStream_t st) {
    k_pme_energy_sum<<<1, 256, 0, st>>>(m, PME_CONV_CTAS, n, out);
}
