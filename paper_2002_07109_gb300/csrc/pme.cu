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
//   fft x3    forward transform along each axis (K log K work per line,
//             FP32): lines of 32 M points (M <= 5) in registers, one warp
//             per line (four neighbouring lines per warp along the strided
//             axes); other lengths a batched mixed-radix (4, 2, 3, 5)
//             Stockham FFT of 16 lines per CTA in shared memory; grid sizes
//             with another prime factor a direct sum per line (K^2 work);
//   convolve  multiply by the influence function B(m) C(m) (FP32 table made
//             on the host in FP64) and accumulate the energy partials
//             sum B C |F(Q)|^2 per CTA (FP64);
//   fft x3    inverse transform (no 1/K normalisation); without the energy,
//             axis 0's forward and inverse transforms and the product are
//             one pass over the grid;
//   gather    per atom, q K/L sum dM M M conv (FP32) plus the removal of the
//             same-molecule pairs, -k q_i q_j erf(beta r)/r, into an FP64
//             gradient (SoA) that the step kernel kicks with.
#include <algorithm>

#include "common.cuh"

namespace {

constexpr int MAX_ORDER = 8;

// M_n(fr + t), t = 0..n-1, and dM_n/dx at the same points, by the recursion
// M_{k+1}(x) = (x M_k(x) + (k + 1 - x) M_k(x - 1)) / k from M_2.
// (The order n is a template parameter so that every array stays in registers.)
template <int n>
__device__ __forceinline__ void bspline_weights(float fr, float* w, float* dw) {
    float a[MAX_ORDER + 1];
#pragma unroll
    for (int t = 0; t <= n; ++t) a[t] = 0.f;
    a[0] = fr;
    a[1] = 1.f - fr;
#pragma unroll
    for (int k = 2; k < n; ++k) {
        if (k == n - 1) {
            // derivative from M_{n-1}: M_n'(fr + t) = M_{n-1}(fr + t) - M_{n-1}(fr + t - 1)
#pragma unroll
            for (int t = 0; t < n; ++t) dw[t] = a[t] - (t > 0 ? a[t - 1] : 0.f);
        }
#pragma unroll
        for (int t = k; t >= 0; --t) {
            const float x = fr + (float)t;
            a[t] = (x * a[t] + ((float)(k + 1) - x) * (t > 0 ? a[t - 1] : 0.f)) / (float)k;
        }
    }
    if (n == 2) {
        dw[0] = 1.f;
        dw[1] = -1.f;
    }
#pragma unroll
    for (int t = 0; t < n; ++t) w[t] = a[t];
}

__device__ __forceinline__ void frac_coord(double x, double iL, int K, int& fl, float& fr) {
    const double f = x * iL;
    const double u = (f - floor(f)) * (double)K;
    double g = floor(u);
    fl = (int)g;
    fr = (float)(u - g);
    if (fl >= K) fl -= K;
}

template <int n>
__global__ void k_pme_spread(DevSys s, DevPme m, int step_off) {
    const int cur = (int)((*s.step_base + step_off) & 1);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < s.n; i += gridDim.x * blockDim.x) {
        int f[3];
        float fr[3];
        frac_coord(s.qx[cur][i], m.iL[0], m.K[0], f[0], fr[0]);
        frac_coord(s.qy[cur][i], m.iL[1], m.K[1], f[1], fr[1]);
        frac_coord(s.qz[cur][i], m.iL[2], m.K[2], f[2], fr[2]);
        float w[3][MAX_ORDER], dw[3][MAX_ORDER];
        #pragma unroll
        for (int d = 0; d < 3; ++d) bspline_weights<n>(fr[d], w[d], dw[d]);
        const float q = s.phi[cur][i].w;
        int ig[3][MAX_ORDER];  // grid index f - t (periodic) of every spline point
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
            for (int t = 0; t < n; ++t) ig[d][t] = f[d] - t < 0 ? f[d] - t + m.K[d] : f[d] - t;
#pragma unroll
        for (int a = 0; a < n; ++a) {
            const float qa = q * w[0][a];
#pragma unroll
            for (int b = 0; b < n; ++b) {
                const float qab = qa * w[1][b];
                const size_t row = ((size_t)ig[0][a] * m.K[1] + ig[1][b]) * m.K[2];
#pragma unroll
                for (int c = 0; c < n; ++c) atomicAdd(&m.qgrid[row + ig[2][c]], fix_round<40>(qab * w[2][c]));
            }
        }
    }
}

__global__ void k_pme_load(DevPme m) {
    const size_t N = (size_t)m.K[0] * m.K[1] * m.K[2];
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < N; k += (size_t)gridDim.x * blockDim.x) {
        const long long v = (long long)m.qgrid[k];
        m.cgrid[k] = make_float2(__ll2float_rn(v) * 9.094947017729282e-13f, 0.f);  // v 2^-40
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

// Batched mixed-radix FFT of the grid lines along one axis: a CTA takes
// FFT_B lines that are neighbours in the grid's fastest other index (so that
// the loads and stores of the strided axes are coalesced), keeps them in
// shared memory and runs the stages of the Stockham autosort formulation
// (each stage reads sub-transforms of span Ns, applies the twiddles
// exp(sign 2 pi i r (j mod Ns) / (Ns R)) and an R-point DFT, and writes its
// outputs in natural order; Govindaraju et al., SC'08), for radices 4, 2, 3
// and 5.  X_k = sum_j x_j exp(sign 2 pi i j k / K), no normalisation.
constexpr int FFT_B = 16;
constexpr int FFT_MAXST = 16;

struct FftPlan {
    int nst;                  // number of stages
    int rad[FFT_MAXST];       // radix of each stage
};

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// sign * i * a
__device__ __forceinline__ float2 cisg(float2 a, float sg) { return make_float2(-sg * a.y, sg * a.x); }

// R-point DFT in place, y_k = sum_r v_r exp(sign 2 pi i r k / R).
__device__ __forceinline__ void small_dft(float2* v, int R, float sg) {
    if (R == 2) {
        const float2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else if (R == 4) {
        const float2 s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
        const float2 s13 = cadd(v[1], v[3]), d13 = cisg(csub(v[1], v[3]), sg);
        v[0] = cadd(s02, s13);
        v[2] = csub(s02, s13);
        v[1] = cadd(d02, d13);
        v[3] = csub(d02, d13);
    } else if (R == 3) {
        const float h = 0.86602540378443865f;  // sin(2 pi / 3)
        const float2 t = cadd(v[1], v[2]), u = cisg(csub(v[1], v[2]), sg * h);
        const float2 m = make_float2(v[0].x - 0.5f * t.x, v[0].y - 0.5f * t.y);
        v[0] = cadd(v[0], t);
        v[1] = cadd(m, u);
        v[2] = csub(m, u);
    } else {  // R == 5
        const float c1 = 0.30901699437494742f, c2 = -0.80901699437494742f;  // cos(2 pi / 5), cos(4 pi / 5)
        const float s1 = 0.95105651629515357f, s2 = 0.58778525229247313f;   // sin(2 pi / 5), sin(4 pi / 5)
        const float2 t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]), t3 = csub(v[1], v[4]), t4 = csub(v[2], v[3]);
        const float2 a0 = v[0];
        const float2 r1 = make_float2(a0.x + c1 * t1.x + c2 * t2.x, a0.y + c1 * t1.y + c2 * t2.y);
        const float2 r2 = make_float2(a0.x + c2 * t1.x + c1 * t2.x, a0.y + c2 * t1.y + c1 * t2.y);
        const float2 i1 = cisg(make_float2(s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y), sg);
        const float2 i2 = cisg(make_float2(s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y), sg);
        v[0] = cadd(a0, cadd(t1, t2));
        v[1] = cadd(r1, i1);
        v[4] = csub(r1, i1);
        v[2] = cadd(r2, i2);
        v[3] = csub(r2, i2);
    }
}

// One Stockham stage of radix R over the FFT_B lines of the CTA.
template <int R>
__device__ __forceinline__ void fft_stage(const float2* src, float2* dst, const float2* tw, int K, int Ns, float sign) {
    const int KR = K / R, tstep = K / (Ns * R);
    for (int t = threadIdx.x; t < FFT_B * KR; t += blockDim.x) {
        const int b = t / KR, j = t - b * KR;
        const float2* x = src + b * K;
        float2* y = dst + b * K;
        float2 v[R];
        const int jm = j % Ns;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float2 a = x[j + r * KR];
            v[r] = r == 0 ? a : cmul(a, tw[r * jm * tstep]);
        }
        small_dft(v, R, sign);
        const int od = (j / Ns) * Ns * R + jm;
#pragma unroll
        for (int r = 0; r < R; ++r) y[od + r * Ns] = v[r];
    }
}

__global__ void k_pme_fft(DevPme m, int axis, float sign, FftPlan pl) {
    extern __shared__ float2 sh[];
    const int K = m.K[axis];
    float2* buf0 = sh;
    float2* buf1 = sh + FFT_B * K;
    float2* tw = sh + 2 * FFT_B * K;
    // lines: index l over the two other axes; element j of line l at base(l) + j stride
    const int nlines = (int)((size_t)m.K[0] * m.K[1] * m.K[2] / K);
    const int l0 = blockIdx.x * FFT_B;
    const int nb = min(FFT_B, nlines - l0);
    size_t stride;
    if (axis == 2) stride = 1;
    else if (axis == 1) stride = m.K[2];
    else stride = (size_t)m.K[1] * m.K[2];
    auto base = [&](int l) -> size_t {
        if (axis == 2) return (size_t)l * m.K[2];
        if (axis == 1) return (size_t)(l / m.K[2]) * m.K[1] * m.K[2] + (l % m.K[2]);
        return (size_t)l;
    };
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        float sn, cs;
        sincospif(2.f * (float)k / (float)K, &sn, &cs);
        tw[k] = make_float2(cs, sign * sn);
    }
    // load: contiguous lines element-fastest, strided lines line-fastest (coalesced either way)
    for (int e = threadIdx.x; e < FFT_B * K; e += blockDim.x) {
        int b, j;
        if (stride == 1) {
            b = e / K;
            j = e - b * K;
        } else {
            j = e / FFT_B;
            b = e - j * FFT_B;
        }
        buf0[b * K + j] = b < nb ? m.cgrid[base(l0 + b) + (size_t)j * stride] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    float2* src = buf0;
    float2* dst = buf1;
    int Ns = 1;
    for (int st = 0; st < pl.nst; ++st) {
        const int R = pl.rad[st];
        if (R == 4) fft_stage<4>(src, dst, tw, K, Ns, sign);
        else if (R == 2) fft_stage<2>(src, dst, tw, K, Ns, sign);
        else if (R == 3) fft_stage<3>(src, dst, tw, K, Ns, sign);
        else fft_stage<5>(src, dst, tw, K, Ns, sign);
        __syncthreads();
        float2* tmp = src;
        src = dst;
        dst = tmp;
        Ns *= R;
    }
    for (int e = threadIdx.x; e < FFT_B * K; e += blockDim.x) {
        int b, j;
        if (stride == 1) {
            b = e / K;
            j = e - b * K;
        } else {
            j = e / FFT_B;
            b = e - j * FFT_B;
        }
        if (b < nb) m.cgrid[base(l0 + b) + (size_t)j * stride] = src[b * K + j];
    }
}

// Radices of an FFT of size K (4s first, then 2, 3, 5); false when K has
// another prime factor (the direct transform serves those sizes).
bool fft_plan(int K, FftPlan& pl) {
    pl.nst = 0;
    int r = K;
    const int rads[4] = {4, 2, 3, 5};
    for (int q : rads)
        while (r % q == 0 && pl.nst < FFT_MAXST) {
            pl.rad[pl.nst++] = q;
            r /= q;
        }
    return r == 1 && K >= 2;
}

// F(Q) <- B C F(Q); energy partial sum B C |F(Q)|^2 of this CTA into eterm.
// ENERGY = false (the steps): the product only, no FP64 energy partials.
template <bool ENERGY>
__global__ void k_pme_convolve(DevPme m) {
    __shared__ double red[256];
    const size_t N = (size_t)m.K[0] * m.K[1] * m.K[2];
    double e = 0.0;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < N; k += (size_t)gridDim.x * blockDim.x) {
        const float2 c = m.cgrid[k];
        const float b = m.bc[k];
        if (ENERGY) e += (double)b * ((double)c.x * c.x + (double)c.y * c.y);
        m.cgrid[k] = make_float2(b * c.x, b * c.y);
    }
    if (!ENERGY) return;
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
template <int n>
__global__ void k_pme_gather(DevSys s, Params p, DevPme m, int step_off) {
    const int cur = (int)((*s.step_base + step_off) & 1);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < s.n; i += gridDim.x * blockDim.x) {
        int f[3];
        float fr[3];
        frac_coord(s.qx[cur][i], m.iL[0], m.K[0], f[0], fr[0]);
        frac_coord(s.qy[cur][i], m.iL[1], m.K[1], f[1], fr[1]);
        frac_coord(s.qz[cur][i], m.iL[2], m.K[2], f[2], fr[2]);
        float w[3][MAX_ORDER], dw[3][MAX_ORDER];
        #pragma unroll
        for (int d = 0; d < 3; ++d) bspline_weights<n>(fr[d], w[d], dw[d]);
        int ig[3][MAX_ORDER];  // grid index f - t (periodic) of every spline point
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
            for (int t = 0; t < n; ++t) ig[d][t] = f[d] - t < 0 ? f[d] - t + m.K[d] : f[d] - t;
        float gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll
        for (int a = 0; a < n; ++a) {
#pragma unroll
            for (int b = 0; b < n; ++b) {
                const size_t row = ((size_t)ig[0][a] * m.K[1] + ig[1][b]) * m.K[2];
                float sx = 0.f, sz = 0.f;
#pragma unroll
                for (int c = 0; c < n; ++c) {
                    const float cv = m.cgrid[row + ig[2][c]].x;
                    sx += cv * w[2][c];
                    sz += cv * dw[2][c];
                }
                gx += dw[0][a] * w[1][b] * sx;
                gy += w[0][a] * dw[1][b] * sx;
                gz += w[0][a] * w[1][b] * sz;
            }
        }
        const float4 hi = s.phi[cur][i], lo = s.plo[cur][i];
        const double kq = KCOUL_D * (double)hi.w;
        double Gx = kq * (double)gx * m.KL[0];
        double Gy = kq * (double)gy * m.KL[1];
        double Gz = kq * (double)gz * m.KL[2];
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

// Lines of K = 32 M points (M = 1..5): one warp per line, no shared-memory
// stages and no barriers.  With n = 32 n1 + n2 and k = k1 + M k2
// (Cooley-Tukey, N1 = M, N2 = 32):
//   X[k1 + M k2] = sum_n2 W_32^(n2 k2) [ W_K^(n2 k1) sum_n1 x[32 n1 + n2] W_M^(n1 k1) ],
// so lane n2 holds x[32 n1 + n2] for n1 < M in registers, takes the M-point
// DFTs in registers, multiplies by the twiddles W_K^(n2 k1), and the warp
// takes the 32-point DFTs across its lanes by shuffles (decimation in
// frequency: 5 butterfly stages, output in bit-reversed lane order).
// Twiddles W_K^e = exp(sign 2 pi i e / K) come from a table in shared memory.
template <int M>
__global__ void __launch_bounds__(256) k_pme_fft_w(DevPme m, int axis, float sign) {
    constexpr int K = 32 * M;
    __shared__ float2 tw[K];
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        float sn, cs;
        sincospif(2.f * (float)k / (float)K, &sn, &cs);
        tw[k] = make_float2(cs, sign * sn);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int nlines = (int)((size_t)m.K[0] * m.K[1] * m.K[2] / K);
    size_t stride;
    if (axis == 2) stride = 1;
    else if (axis == 1) stride = m.K[2];
    else stride = (size_t)m.K[1] * m.K[2];
    const int rev = (int)(__brev((unsigned)lane) >> 27);
    for (int l = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); l < nlines; l += gridDim.x * (blockDim.x >> 5)) {
        size_t b0;
        if (axis == 2) b0 = (size_t)l * m.K[2];
        else if (axis == 1) b0 = (size_t)(l / m.K[2]) * m.K[1] * m.K[2] + (l % m.K[2]);
        else b0 = (size_t)l;
        float2 v[M > 1 ? M : 2];
#pragma unroll
        for (int n1 = 0; n1 < M; ++n1) v[n1] = m.cgrid[b0 + (size_t)(32 * n1 + lane) * stride];
        if (M > 1) small_dft(v, M, sign);
#pragma unroll
        for (int k1 = 1; k1 < M; ++k1) v[k1] = cmul(v[k1], tw[(lane * k1) % K]);
#pragma unroll
        for (int sh = 16; sh > 0; sh >>= 1) {
            const bool low = (lane & sh) != 0;
            const float2 w = tw[(lane & (sh - 1)) * (K / (2 * sh))];
#pragma unroll
            for (int k1 = 0; k1 < M; ++k1) {
                float2 b;
                b.x = __shfl_xor_sync(0xffffffffu, v[k1].x, sh);
                b.y = __shfl_xor_sync(0xffffffffu, v[k1].y, sh);
                v[k1] = low ? cmul(csub(b, v[k1]), w) : cadd(v[k1], b);
            }
        }
#pragma unroll
        for (int k1 = 0; k1 < M; ++k1) m.cgrid[b0 + (size_t)(k1 + M * rev) * stride] = v[k1];
    }
}

// The transforms of four lines of K = 32 M points held by one warp (lane n2
// holds x[32 n1 + n2] of each line for n1 < M): M-point DFTs in registers,
// twiddles W_K^(n2 k1) from tw, then the 32-point DFTs across the lanes by
// shuffles.  On return lane l holds X[k1 + M rev(l)] of each line (rev: the
// 5-bit reversal of l).
template <int M>
__device__ __forceinline__ void warp_fft4(float2 (&v)[4][M > 1 ? M : 2], const float2* tw, int lane, float sign) {
    constexpr int K = 32 * M;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (M > 1) small_dft(v[q], M, sign);
#pragma unroll
        for (int k1 = 1; k1 < M; ++k1) v[q][k1] = cmul(v[q][k1], tw[(lane * k1) % K]);
    }
#pragma unroll
    for (int sh = 16; sh > 0; sh >>= 1) {
        const bool low = (lane & sh) != 0;
        const float2 w = tw[(lane & (sh - 1)) * (K / (2 * sh))];
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int k1 = 0; k1 < M; ++k1) {
                float2 b;
                b.x = __shfl_xor_sync(0xffffffffu, v[q][k1].x, sh);
                b.y = __shfl_xor_sync(0xffffffffu, v[q][k1].y, sh);
                v[q][k1] = low ? cmul(csub(b, v[q][k1]), w) : cadd(v[q][k1], b);
            }
    }
}

// The same transform for four neighbouring lines of a strided axis (axis 0
// or 1: lines l..l+3 are neighbours along the contiguous axis), one warp for
// all four: each lane loads and stores 32 contiguous bytes (four complex
// values) per point instead of 8, so the strided passes use whole sectors.
template <int M>
__global__ void __launch_bounds__(256) k_pme_fft_w4(DevPme m, int axis, float sign) {
    constexpr int K = 32 * M;
    __shared__ float2 tw[K];
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        float sn, cs;
        sincospif(2.f * (float)k / (float)K, &sn, &cs);
        tw[k] = make_float2(cs, sign * sn);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int ngroups = (int)((size_t)m.K[0] * m.K[1] * m.K[2] / K / 4);
    const size_t stride = axis == 1 ? (size_t)m.K[2] : (size_t)m.K[1] * m.K[2];
    const int rev = (int)(__brev((unsigned)lane) >> 27);
    for (int g = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); g < ngroups; g += gridDim.x * (blockDim.x >> 5)) {
        const int l = 4 * g;
        const size_t b0 = axis == 1 ? (size_t)(l / m.K[2]) * m.K[1] * m.K[2] + (l % m.K[2]) : (size_t)l;
        float2 v[4][M > 1 ? M : 2];
#pragma unroll
        for (int n1 = 0; n1 < M; ++n1) {
            const float4* src = reinterpret_cast<const float4*>(m.cgrid + b0 + (size_t)(32 * n1 + lane) * stride);
            const float4 a = src[0], b = src[1];
            v[0][n1] = make_float2(a.x, a.y);
            v[1][n1] = make_float2(a.z, a.w);
            v[2][n1] = make_float2(b.x, b.y);
            v[3][n1] = make_float2(b.z, b.w);
        }
        warp_fft4<M>(v, tw, lane, sign);
#pragma unroll
        for (int k1 = 0; k1 < M; ++k1) {
            float4* dst = reinterpret_cast<float4*>(m.cgrid + b0 + (size_t)(k1 + M * rev) * stride);
            dst[0] = make_float4(v[0][k1].x, v[0][k1].y, v[1][k1].x, v[1][k1].y);
            dst[1] = make_float4(v[2][k1].x, v[2][k1].y, v[3][k1].x, v[3][k1].y);
        }
    }
}

// Axis 0 of the forward transform, the influence function and axis 0 of
// the inverse transform in one pass (evaluations without the energy): each
// warp transforms four neighbouring lines along axis 0 as k_pme_fft_w4,
// multiplies every point by B C (k_pme_convolve's product, the same
// rounding), brings the lines back to natural order through shared memory
// and transforms them back, so that the grid is read and written once for
// the three steps.
template <int M>
__global__ void __launch_bounds__(256) k_pme_conv_x4(DevPme m) {
    constexpr int K = 32 * M;
    __shared__ float2 twf[K], twi[K];
    __shared__ float2 sl[8][4][K];
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        float sn, cs;
        sincospif(2.f * (float)k / (float)K, &sn, &cs);
        twf[k] = make_float2(cs, -sn);
        twi[k] = make_float2(cs, sn);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const int ngroups = (int)((size_t)m.K[1] * m.K[2] / 4);
    const size_t stride = (size_t)m.K[1] * m.K[2];
    const int rev = (int)(__brev((unsigned)lane) >> 27);
    for (int g = blockIdx.x * (blockDim.x >> 5) + wl; g < ngroups; g += gridDim.x * (blockDim.x >> 5)) {
        const size_t b0 = 4 * (size_t)g;
        float2 v[4][M > 1 ? M : 2];
#pragma unroll
        for (int n1 = 0; n1 < M; ++n1) {
            const float4* src = reinterpret_cast<const float4*>(m.cgrid + b0 + (size_t)(32 * n1 + lane) * stride);
            const float4 a = src[0], b = src[1];
            v[0][n1] = make_float2(a.x, a.y);
            v[1][n1] = make_float2(a.z, a.w);
            v[2][n1] = make_float2(b.x, b.y);
            v[3][n1] = make_float2(b.z, b.w);
        }
        warp_fft4<M>(v, twf, lane, -1.f);
        __syncwarp();
#pragma unroll
        for (int k1 = 0; k1 < M; ++k1) {
            const int kx = k1 + M * rev;
            const float4 bc = *reinterpret_cast<const float4*>(m.bc + b0 + (size_t)kx * stride);
            sl[wl][0][kx] = make_float2(bc.x * v[0][k1].x, bc.x * v[0][k1].y);
            sl[wl][1][kx] = make_float2(bc.y * v[1][k1].x, bc.y * v[1][k1].y);
            sl[wl][2][kx] = make_float2(bc.z * v[2][k1].x, bc.z * v[2][k1].y);
            sl[wl][3][kx] = make_float2(bc.w * v[3][k1].x, bc.w * v[3][k1].y);
        }
        __syncwarp();
#pragma unroll
        for (int n1 = 0; n1 < M; ++n1)
#pragma unroll
            for (int q = 0; q < 4; ++q) v[q][n1] = sl[wl][q][32 * n1 + lane];
        warp_fft4<M>(v, twi, lane, 1.f);
#pragma unroll
        for (int k1 = 0; k1 < M; ++k1) {
            float4* dst = reinterpret_cast<float4*>(m.cgrid + b0 + (size_t)(k1 + M * rev) * stride);
            dst[0] = make_float4(v[0][k1].x, v[0][k1].y, v[1][k1].x, v[1][k1].y);
            dst[1] = make_float4(v[2][k1].x, v[2][k1].y, v[3][k1].x, v[3][k1].y);
        }
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

void launch_pme(const DevSys& s, const Params& p, const DevPme& m, int step_off, cudaStream_t st, bool energy) {
    const int tb = 128;
    const int nb = (s.n + tb - 1) / tb;
    switch (m.order) {
        case 3: k_pme_spread<3><<<nb, tb, 0, st>>>(s, m, step_off); break;
        case 4: k_pme_spread<4><<<nb, tb, 0, st>>>(s, m, step_off); break;
        case 5: k_pme_spread<5><<<nb, tb, 0, st>>>(s, m, step_off); break;
        case 6: k_pme_spread<6><<<nb, tb, 0, st>>>(s, m, step_off); break;
        case 7: k_pme_spread<7><<<nb, tb, 0, st>>>(s, m, step_off); break;
        default: k_pme_spread<8><<<nb, tb, 0, st>>>(s, m, step_off); break;
    }
    const size_t N = (size_t)m.K[0] * m.K[1] * m.K[2];
    k_pme_load<<<(int)std::min<size_t>((N + 255) / 256, 4096), 256, 0, st>>>(m);
    const int lines[3] = {m.K[1] * m.K[2], m.K[0] * m.K[2], m.K[0] * m.K[1]};
    auto transform = [&](int axis, float sign) {
        FftPlan pl;
        const int K = m.K[axis], Mw = K / 32, nl = lines[axis];
        const int wb = std::min((nl + 7) / 8, 152 * 8);
        // four lines per warp along a strided axis (lines grouped by four
        // along the contiguous axis, 32-byte aligned)
        const bool four = axis != 2 && m.K[2] % 4 == 0;
        const int wb4 = std::min((nl / 4 + 7) / 8, 152 * 8);
        if (four && K % 32 == 0 && Mw >= 1 && Mw <= 5) {
            if (Mw == 1) k_pme_fft_w4<1><<<wb4, 256, 0, st>>>(m, axis, sign);
            else if (Mw == 2) k_pme_fft_w4<2><<<wb4, 256, 0, st>>>(m, axis, sign);
            else if (Mw == 3) k_pme_fft_w4<3><<<wb4, 256, 0, st>>>(m, axis, sign);
            else if (Mw == 4) k_pme_fft_w4<4><<<wb4, 256, 0, st>>>(m, axis, sign);
            else k_pme_fft_w4<5><<<wb4, 256, 0, st>>>(m, axis, sign);
        } else if (K % 32 == 0 && Mw >= 1 && Mw <= 5) {
            if (Mw == 1) k_pme_fft_w<1><<<wb, 256, 0, st>>>(m, axis, sign);
            else if (Mw == 2) k_pme_fft_w<2><<<wb, 256, 0, st>>>(m, axis, sign);
            else if (Mw == 3) k_pme_fft_w<3><<<wb, 256, 0, st>>>(m, axis, sign);
            else if (Mw == 4) k_pme_fft_w<4><<<wb, 256, 0, st>>>(m, axis, sign);
            else k_pme_fft_w<5><<<wb, 256, 0, st>>>(m, axis, sign);
        } else if (fft_plan(m.K[axis], pl)) {
            const size_t smem = (2 * (size_t)FFT_B + 1) * m.K[axis] * sizeof(float2);
            k_pme_fft<<<(lines[axis] + FFT_B - 1) / FFT_B, 128, smem, st>>>(m, axis, sign, pl);
        } else {
            k_pme_dft<<<lines[axis], 128, 2 * m.K[axis] * sizeof(float2), st>>>(m, axis, sign);
        }
    };
    // without the energy, axis 0's two transforms and the product in one
    // pass when its lines are 32 M points that four-line warps take
    const int M0 = m.K[0] / 32;
    const bool fuse = !energy && m.K[0] % 32 == 0 && M0 >= 1 && M0 <= 5 && m.K[2] % 4 == 0;
    if (fuse) {
        transform(2, -1.f);
        transform(1, -1.f);
        const int wb = std::min((lines[0] / 4 + 7) / 8, 152 * 8);
        if (M0 == 1) k_pme_conv_x4<1><<<wb, 256, 0, st>>>(m);
        else if (M0 == 2) k_pme_conv_x4<2><<<wb, 256, 0, st>>>(m);
        else if (M0 == 3) k_pme_conv_x4<3><<<wb, 256, 0, st>>>(m);
        else if (M0 == 4) k_pme_conv_x4<4><<<wb, 256, 0, st>>>(m);
        else k_pme_conv_x4<5><<<wb, 256, 0, st>>>(m);
        transform(1, 1.f);
        transform(2, 1.f);
    } else {
        for (int axis = 2; axis >= 0; --axis) transform(axis, -1.f);
        if (energy) k_pme_convolve<true><<<PME_CONV_CTAS, 256, 0, st>>>(m);
        else k_pme_convolve<false><<<PME_CONV_CTAS, 256, 0, st>>>(m);
        for (int axis = 2; axis >= 0; --axis) transform(axis, 1.f);
    }
    switch (m.order) {
        case 3: k_pme_gather<3><<<nb, tb, 0, st>>>(s, p, m, step_off); break;
        case 4: k_pme_gather<4><<<nb, tb, 0, st>>>(s, p, m, step_off); break;
        case 5: k_pme_gather<5><<<nb, tb, 0, st>>>(s, p, m, step_off); break;
        case 6: k_pme_gather<6><<<nb, tb, 0, st>>>(s, p, m, step_off); break;
        case 7: k_pme_gather<7><<<nb, tb, 0, st>>>(s, p, m, step_off); break;
        default: k_pme_gather<8><<<nb, tb, 0, st>>>(s, p, m, step_off); break;
    }
}

void launch_pme_energy(const DevPme& m, int n, double* out, cudaStream_t st) {
    k_pme_energy_sum<<<1, 256, 0, st>>>(m, PME_CONV_CTAS, n, out);
}
