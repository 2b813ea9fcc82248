// C ABI of the BOUNCE library (declared in include/bounce.h): context
// management, host-side set-up (topology tables, the jump bounds
// L_ab = sup |chi W'_ab| of Sec. IV.A, the cell grid) and the run loop,
// which replays CUDA graphs of captured chunks of steps.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/bounce.h"
#include "common.cuh"

void nlist_set_smem_limit(size_t bytes);
int diff_param_count();
void launch_pair_forward(const DevSys& s, const Params& p, const float* qt, const float* sig, const float* eps, int T,
                         int cur, double* F, double* eatom, double* esum, cudaStream_t st);
void launch_pair_backward(const DevSys& s, const Params& p, const float* qt, const float* sig, const float* eps, int T,
                          int cur, const double* U, double w, double* gpos, double* part, double* psum,
                          cudaStream_t st);
void launch_pair_hist(const DevSys& s, const Params& p, int cur, int ta, int tb, double r_max, int n_bins,
                      unsigned long long* hist, cudaStream_t st);
void launch_msd(const DevSys& s, const double* rx, const double* ry, const double* rz, int cur, int t,
                double* terms, cudaStream_t st);

namespace {

constexpr int CHUNK = 32;  // steps per captured graph

struct Buf {
    void* p = nullptr;
    size_t bytes = 0;
};

}  // namespace

struct bounce_ctx {
    bounce_config cfg{};
    std::string err;
    int n = 0;
    bool have_topo = false, have_lj = false, have_state = false;
    // host copies
    std::vector<int> type, mol;
    std::vector<double> mass, charge;
    std::vector<int> bt_off;
    std::vector<int4> bt_idx;
    std::vector<float2> bt_par;
    int n_types = 0;
    double L[BOUNCE_MAXT * BOUNCE_MAXT] = {0};
    double Lstar[BOUNCE_MAXT] = {0};
    long long step0 = 0;
    bool have_msd_ref = false;
    // device
    std::vector<Buf> bufs;
    DevSys ds{};
    Params pp{};
    double* terms = nullptr;     // energy scratch [6 n]
    double* msd_ref = nullptr;   // [3 n] reference positions of bounce_msd
    unsigned long long* hist = nullptr;
    int hist_alloc = 0;
    long long* d_step = nullptr;
    int* h_err = nullptr;        // pinned
    double* h_stage = nullptr;   // pinned [6 n]: interleaved q then v on their way to or from the device
    double* d_stage = nullptr;   // device [6 n]
    unsigned long long* h_cnt = nullptr;
    int bitmap_warps = 1;        // window words per bitmap of the row builder
    size_t bitmap_bytes = 0;     // its shared memory per CTA
    int ncell_alloc = 0;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph[5][64] = {};  // [integrator][RESPA phase of the chunk's first step]
    long long cur_step = 0;              // host mirror of the device step counter
    bool rows_valid = false;             // rows were requested for this topology and replica layout
    bool has_pme = false;
    DevPme pme{};
    double* diff_part = nullptr;   // [NPAR n + NPAR] parameter partials and sums of the pair backward
    double e_self = 0.0;
    // cluster-pair path: allocated capacities (buffers grow, never shrink)
    int cl_cap_ncol = 0, cl_cap_ncl = 0, cl_cap_items = 0;
    size_t cl_cap_lst[2] = {0, 0};
    bool cl_atoms_alloc = false;
    // after BAOAB runs on clusters the step kernel did not test the rows:
    // the next row consumer tests the displacement first
    bool rows_check_due = false;
    bool rows_partial = false;    // a run left the rows of atoms with L* = 0 empty (ROWS_ACTIVE)
    // jump rows that keep only the partners a jump can draw (LJ alone on the
    // jumps, one bound per type): the rows buffers then hold the jump step's
    // rows, and the entry points that read every row get full rows in a
    // second set of buffers, so that reading leaves the run's rows alone
    bool jfilter = false;
    unsigned jmove = ~0u;         // types whose displacement can change a jump row
    int rows_kind = 0;            // what the rows buffers hold: 0 nothing usable, 1 full rows, 2 jump rows
    bool rows_swapped = false;    // ds.rows / ds.nlong point at the readers' buffers
    int* rows_main = nullptr;     // the run's buffers while swapped
    int* nlong_main = nullptr;
    int* rows_alt = nullptr;      // the readers' buffers (allocated on first use)
    int* nlong_alt = nullptr;
    long long pos_version = 0;    // bumped whenever the positions change
    long long reader_version = -1;  // positions the readers' rows were built at
    int* d_act_order = nullptr;   // device copy of DevSys::act_order
    // tuning (bounce_autotune): cluster column edge factor, tile j-block and grid
    double cl_edge_factor = 1.0;
    bool cl_force = false;        // the next setup_clusters recomputes the grid
    int tile_j = 64, tile_blocks = 152 * 4;
    int4* tile_items = nullptr;
    int tile_cap = 0;
    std::vector<int> rep_bounds;  // [replicas + 1] atom ranges for the tiles ({0, n} for one system)
    bool lite_jumps = false;      // BOUNCE integrators take the thread-per-atom step kernel
};

namespace {

int fail(bounce_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg;
    return code;
}

#define CU(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(c, BOUNCE_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

template <class T>
int dalloc(bounce_ctx* c, T** out, size_t count) {
    void* p = nullptr;
    size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) return fail(c, BOUNCE_ERR_CUDA, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    cudaMemset(p, 0, bytes);
    c->bufs.push_back({p, bytes});
    *out = (T*)p;
    return BOUNCE_OK;
}

void drop_graphs(bounce_ctx* c) {
    for (auto& row : c->graph)
        for (auto& g : row)
            if (g) {
                cudaGraphExecDestroy(g);
                g = nullptr;
            }
}

void reset_cluster_caps(bounce_ctx* c) {
    c->cl_cap_ncol = c->cl_cap_ncl = c->cl_cap_items = 0;
    c->cl_cap_lst[0] = c->cl_cap_lst[1] = 0;
    c->cl_atoms_alloc = false;
    c->rows_check_due = false;
}

void free_all(bounce_ctx* c) {
    if (c->h_stage) cudaFreeHost(c->h_stage);
    c->h_stage = nullptr;
    drop_graphs(c);
    for (auto& b : c->bufs) cudaFree(b.p);
    c->bufs.clear();
    c->ds = DevSys{};
    c->terms = nullptr;
    c->d_step = nullptr;
    c->msd_ref = nullptr;
    c->hist = nullptr;
    c->hist_alloc = 0;
    c->have_msd_ref = false;
    c->has_pme = false;
    c->pme = DevPme{};
    c->diff_part = nullptr;
    c->tile_items = nullptr;
    c->tile_cap = 0;
    c->d_act_order = nullptr;
    c->rows_partial = false;
    c->rows_kind = 0;
    c->rows_swapped = false;
    c->rows_main = c->nlong_main = c->rows_alt = c->nlong_alt = nullptr;
    c->reader_version = -1;
    reset_cluster_caps(c);
}

// ---------------------------------------------------------------- bounds
double chi_host(double r, double on, double off) {
    if (!(off > on)) return r >= off ? 1.0 : 0.0;
    double s = std::min(std::max((r - on) / (off - on), 0.0), 1.0);
    return s * s * s * (10.0 + s * (-15.0 + 6.0 * s));
}

double dW_host(double r, double qq, double sig, double eps, double beta) {
    double w;
    if (beta > 0) w = -KCOUL_D * qq * (std::erfc(beta * r) / (r * r) + 2.0 * beta / std::sqrt(M_PI) * std::exp(-beta * beta * r * r) / r);
    else w = -KCOUL_D * qq / (r * r);
    if (eps != 0.0) {
        double sr6 = std::pow(sig / r, 6);
        w += -24.0 * eps * (2.0 * sr6 * sr6 - sr6) / r;
    }
    return w;
}

// sup over r in [r', r_c) of |chi(r) W'(r)|: grid scan, then golden-section
// refinement of the best bracket.
double sup_chi_dW(const bounce_config& cfg, double qq, double sig, double eps) {
    const double lo = cfg.r_off > cfg.r_on ? cfg.r_on : cfg.r_off;
    const bool cut = std::isfinite(cfg.r_cut) && cfg.r_cut > 0;
    const double hi = cut ? cfg.r_cut : cfg.r_off + 60.0;
    if (!(hi > lo)) return 0.0;
    auto f = [&](double r) {
        if (cut && !(r < cfg.r_cut)) return 0.0;
        return std::fabs(chi_host(r, cfg.r_on, cfg.r_off) * dW_host(r, qq, sig, eps, cfg.ewald_beta));
    };
    const int N = 400000;
    const double h = (hi - lo) / N;
    int kbest = 0;
    double best = -1.0;
    for (int k = 0; k <= N; ++k) {
        double v = f(lo + k * h);
        if (v > best) {
            best = v;
            kbest = k;
        }
    }
    double a = lo + std::max(kbest - 2, 0) * h, b = lo + std::min(kbest + 2, N) * h;
    const double g = 0.5 * (std::sqrt(5.0) - 1.0);
    double x1 = b - g * (b - a), x2 = a + g * (b - a), f1 = f(x1), f2 = f(x2);
    for (int it = 0; it < 200 && b - a > 1e-13; ++it) {
        if (f1 > f2) {
            b = x2;
            x2 = x1;
            f2 = f1;
            x1 = b - g * (b - a);
            f1 = f(x1);
        } else {
            a = x1;
            x1 = x2;
            f1 = f2;
            x2 = a + g * (b - a);
            f2 = f(x2);
        }
    }
    return std::max(best, std::max(f1, f2));
}

void compute_bounds(bounce_ctx* c, const std::vector<double>& sig, const std::vector<double>& eps) {
    const int T = c->n_types;
    double qmin[BOUNCE_MAXT], qmax[BOUNCE_MAXT];
    bool present[BOUNCE_MAXT] = {false};
    for (int t = 0; t < T; ++t) qmin[t] = qmax[t] = 0.0;
    for (int i = 0; i < c->n; ++i) {
        int t = c->type[i];
        double q = c->charge[i];
        if (!present[t]) {
            qmin[t] = qmax[t] = q;
            present[t] = true;
        } else {
            qmin[t] = std::min(qmin[t], q);
            qmax[t] = std::max(qmax[t], q);
        }
    }
    for (int a = 0; a < BOUNCE_MAXT; ++a) c->Lstar[a] = 0.0;
    for (int a = 0; a < T; ++a)
        for (int b = 0; b < T; ++b) {
            double best = 0.0;
            const double qa[2] = {qmin[a], qmax[a]}, qb[2] = {qmin[b], qmax[b]};
            for (int x = 0; x < 2; ++x)
                for (int y = 0; y < 2; ++y)
                    best = std::max(best, sup_chi_dW(c->cfg, c->cfg.jump_coulomb ? qa[x] * qb[y] : 0.0,
                                                     sig[a * T + b], eps[a * T + b]));
            c->L[a * T + b] = best * (1.0 + 1e-6);
            c->Lstar[a] = std::max(c->Lstar[a], c->L[a * T + b]);
        }
}

bool finite_cut(const bounce_config& g) { return std::isfinite(g.r_cut) && g.r_cut > 0; }

// Short candidate rows (r < r_off + skin) for F_0 exist only for systems
// without a cutoff (all pairs); with a cutoff the pair sums run over clusters.
bool short_rows(const bounce_config& g) {
    const double rs = g.r_off + g.skin;
    return g.jump_coulomb && std::isfinite(rs) && !finite_cut(g);
}

double r_list(const bounce_config& cfg) {
    const bool cut = std::isfinite(cfg.r_cut) && cfg.r_cut > 0;
    return cut ? cfg.r_cut + cfg.skin : INFINITY;
}

// ------------------------------------------------------------- SPME set-up
double bspline_host(double x, int n) {
    if (n == 2) return (x >= 0.0 && x <= 2.0) ? 1.0 - std::fabs(x - 1.0) : 0.0;
    return (x * bspline_host(x, n - 1) + (n - x) * bspline_host(x - 1.0, n - 1)) / (n - 1);
}

// |b(m)|^2 of the Euler exponential spline; at the zero of odd orders
// (m = K/2) the mean of the two neighbours.
std::vector<double> bmod2_host(int K, int n) {
    std::vector<double> s(K), out(K);
    for (int m = 0; m < K; ++m) {
        double re = 0.0, im = 0.0;
        for (int k = 0; k <= n - 2; ++k) {
            const double w = bspline_host(k + 1.0, n), a = 2.0 * M_PI * m * k / K;
            re += w * std::cos(a);
            im += w * std::sin(a);
        }
        s[m] = re * re + im * im;
    }
    for (int m = 0; m < K; ++m)
        out[m] = s[m] > 1e-7 ? 1.0 / s[m] : 0.5 * (1.0 / s[(m - 1 + K) % K] + 1.0 / s[(m + 1) % K]);
    return out;
}

int setup_pme(bounce_ctx* c) {
    const bounce_config& g = c->cfg;
    c->has_pme = false;
    if (!(g.periodic && g.ewald_beta > 0 && g.pme_grid[0] > 0 && g.pme_grid[1] > 0 && g.pme_grid[2] > 0)) return BOUNCE_OK;
    if (g.pme_order < 3 || g.pme_order > 8 || g.pme_grid[0] > 512 || g.pme_grid[1] > 512 || g.pme_grid[2] > 512 ||
        g.respa_m < 1 || g.respa_m > 8)
        return fail(c, BOUNCE_ERR_INVALID_ARG, "bad SPME or RESPA parameters");
    DevPme& m = c->pme;
    for (int d = 0; d < 3; ++d) {
        m.K[d] = g.pme_grid[d];
        m.L[d] = g.box[d];
        m.iL[d] = 1.0 / g.box[d];
        m.KL[d] = (double)m.K[d] / g.box[d];
        if (m.K[d] < g.pme_order) return fail(c, BOUNCE_ERR_INVALID_ARG, "SPME grid smaller than the order");
    }
    m.order = g.pme_order;
    m.beta = (float)g.ewald_beta;
    m.two_b_sqrtpi = (float)(2.0 * g.ewald_beta / std::sqrt(M_PI));
    const size_t N = (size_t)m.K[0] * m.K[1] * m.K[2];
    // influence function B(m) C(m), C = exp(-pi^2 m^2/beta^2)/(pi V m^2), in FP64
    const double V = g.box[0] * g.box[1] * g.box[2];
    std::vector<double> b[3];
    for (int d = 0; d < 3; ++d) b[d] = bmod2_host(m.K[d], m.order);
    std::vector<float> bc(N);
    for (int i = 0; i < m.K[0]; ++i) {
        const double fx = (i <= m.K[0] / 2 ? i : i - m.K[0]) / g.box[0];
        for (int j = 0; j < m.K[1]; ++j) {
            const double fy = (j <= m.K[1] / 2 ? j : j - m.K[1]) / g.box[1];
            for (int k = 0; k < m.K[2]; ++k) {
                const double fz = (k <= m.K[2] / 2 ? k : k - m.K[2]) / g.box[2];
                const double m2 = fx * fx + fy * fy + fz * fz;
                const double C = m2 > 0 ? std::exp(-M_PI * M_PI * m2 / (g.ewald_beta * g.ewald_beta)) / (M_PI * V * m2) : 0.0;
                bc[((size_t)i * m.K[1] + j) * m.K[2] + k] = (float)(b[0][i] * b[1][j] * b[2][k] * C);
            }
        }
    }
    // same-molecule partners of every atom
    std::vector<int> off(c->n + 1, 0), idx;
    {
        std::vector<std::vector<int>> bym;
        int maxm = 0;
        for (int i = 0; i < c->n; ++i) maxm = std::max(maxm, c->mol[i] + 1);
        bym.resize(maxm);
        for (int i = 0; i < c->n; ++i) bym[c->mol[i]].push_back(i);
        for (int i = 0; i < c->n; ++i) {
            for (int j : bym[c->mol[i]])
                if (j != i) idx.push_back(j);
            off[i + 1] = (int)idx.size();
        }
    }
    float* dbc;
    int *doff, *didx;
    int r;
    if ((r = dalloc(c, &m.qgrid, N)) || (r = dalloc(c, &m.cgrid, N)) || (r = dalloc(c, &dbc, N)) ||
        (r = dalloc(c, &m.grad, 3 * (size_t)c->n)) || (r = dalloc(c, &m.eexcl, c->n)) || (r = dalloc(c, &m.eterm, 256)) ||
        (r = dalloc(c, &doff, c->n + 1)) || (r = dalloc(c, &didx, std::max<size_t>(idx.size(), 1))))
        return r;
    CU(cudaMemcpy(dbc, bc.data(), N * sizeof(float), cudaMemcpyHostToDevice));
    CU(cudaMemcpy(doff, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice));
    if (!idx.empty()) CU(cudaMemcpy(didx, idx.data(), idx.size() * sizeof(int), cudaMemcpyHostToDevice));
    m.bc = dbc;
    m.ex_off = doff;
    m.ex_idx = didx;
    c->ds.grecip = m.grad;
    double q2 = 0.0;
    for (int i = 0; i < c->n; ++i) q2 += c->charge[i] * c->charge[i];
    c->e_self = -KCOUL_D * g.ewald_beta / std::sqrt(M_PI) * q2;
    c->has_pme = true;
    return BOUNCE_OK;
}

void fill_params(bounce_ctx* c, const std::vector<double>& sig, const std::vector<double>& eps) {
    Params& p = c->pp;
    const bounce_config& g = c->cfg;
    const int T = c->n_types;
    for (int k = 0; k < BOUNCE_MAXT * BOUNCE_MAXT; ++k) p.c12[k] = p.c6[k] = 0.f;
    for (int a = 0; a < T; ++a)
        for (int b = 0; b < T; ++b) {
            double s6 = std::pow(sig[a * T + b], 6);
            p.c12[a * BOUNCE_MAXT + b] = (float)(4.0 * eps[a * T + b] * s6 * s6);
            p.c6[a * BOUNCE_MAXT + b] = (float)(4.0 * eps[a * T + b] * s6);
        }
    p.kcoul = (float)KCOUL_D;
    const bool cut = std::isfinite(g.r_cut) && g.r_cut > 0;
    const double rc2 = cut ? g.r_cut * g.r_cut : INFINITY;
    p.rc2_lo = cut ? (float)(rc2 * (1.0 - 1e-5)) : INFINITY;
    p.rc2_hi = cut ? (float)(rc2 * (1.0 + 1e-5)) : INFINITY;
    p.rc2_d = rc2;
    p.chi_step = g.r_off > g.r_on ? 0 : 1;
    p.r_on = (float)g.r_on;
    p.r_off = (float)g.r_off;
    p.inv_span = g.r_off > g.r_on ? (float)(1.0 / (g.r_off - g.r_on)) : 0.f;
    p.ebeta = (float)g.ewald_beta;
    p.e2b_sqrtpi = (float)(2.0 * g.ewald_beta / std::sqrt(M_PI));
    p.periodic = g.periodic;
    for (int d = 0; d < 3; ++d) {
        double Lb = g.periodic ? g.box[d] : 1.0;
        p.Ld[d] = Lb;
        p.iLd[d] = 1.0 / Lb;
        p.Lhi[d] = (float)Lb;
        p.Llo[d] = (float)(Lb - (double)p.Lhi[d]);
        p.invL[d] = (float)(1.0 / Lb);
    }
    const double rl = r_list(g);
    const double rl2 = rl * rl;
    p.rlist2_d = rl2;
    p.rlist2_lo = std::isfinite(rl2) ? (float)(rl2 * (1.0 - 1e-5)) : INFINITY;
    p.rlist2_hi = std::isfinite(rl2) ? (float)(rl2 * (1.0 + 1e-5)) : INFINITY;
    const double rs = g.r_off + g.skin;
    p.rshort2 = short_rows(g) ? (float)(rs * rs * (1.0 + 1e-4)) : INFINITY;
    p.coul_jump = g.jump_coulomb ? 1 : 0;
    p.typed = g.pair_bounds ? 1 : 0;
    p.n_types = T;
    for (int k = 0; k < BOUNCE_MAXT * BOUNCE_MAXT; ++k) {
        p.lq[k] = 0u;
        p.lq_m[k] = 0u;
        p.lq_s[k] = 0u;
        p.lt_d[k] = 0.0;
    }
    for (int a = 0; a < T; ++a)
        for (int b = 0; b < T; ++b) {
            const double L = c->L[a * T + b];
            if (L > 0.0) {
                const double q = std::ceil(L / c->Lstar[a] * 65536.0) + 1.0;
                p.lq[a * BOUNCE_MAXT + b] = (uint32_t)q;
                p.lt_d[a * BOUNCE_MAXT + b] = (q * c->Lstar[a]) * (1.0 / 65536.0);
                // division by the invariant d = Lq_ab >= 2 (Granlund and Montgomery 1994, Fig. 4.1):
                // l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1, x / d = (t + ((x - t) >> 1)) >> (l - 1)
                const uint64_t d = (uint64_t)q;
                int l = 0;
                while ((1ull << l) < d) ++l;
                p.lq_m[a * BOUNCE_MAXT + b] = (uint32_t)(((1ull << 32) * ((1ull << l) - d)) / d + 1);
                p.lq_s[a * BOUNCE_MAXT + b] = (uint32_t)(l - 1);
            }
        }
    for (int a = 0; a < BOUNCE_MAXT; ++a) {
        p.Lstar_d[a] = c->Lstar[a];
        p.Lstar_f[a] = (float)c->Lstar[a];
    }
    p.beta = 1.0 / (KB_D * g.temperature_K);
    p.dt = g.dt_fs;
    p.beta_f = (float)p.beta;
    p.dt_half_f = (float)(0.5 * p.dt);
    p.c1 = std::exp(-g.gamma_per_fs * g.dt_fs);
    p.skin_half2 = std::isfinite(rl) ? 0.25 * g.skin * g.skin : INFINITY;
    p.key0 = (uint32_t)(g.seed & 0xFFFFFFFFull);
    p.key1 = (uint32_t)(g.seed >> 32);
}

// Cell grid for the current host positions: cells of edge >= r_list / 3
// (the row builder scans, for each (y, z) cell row within reach, only the
// x-span of cells the r_list sphere can touch).
int setup_grid(bounce_ctx* c, const double* q) {
    DevSys& s = c->ds;
    const double rl = r_list(c->cfg);
    const double reach = std::isfinite(rl) ? rl * (1.0 + 1e-5) + 1e-3 : INFINITY;
    const double edge_min = reach / 3.0;
    int nc[3] = {1, 1, 1}, m[3] = {0, 0, 0};
    float org[3] = {0.f, 0.f, 0.f}, ih[3] = {0.f, 0.f, 0.f}, hh[3] = {1.f, 1.f, 1.f};
    for (int d = 0; d < 3; ++d) {
        double h = 1.0;
        if (c->cfg.periodic) {
            const double Lb = c->cfg.box[d];
            nc[d] = std::isfinite(edge_min) ? std::max(1, (int)std::floor(Lb / edge_min)) : 1;
            nc[d] = std::min(nc[d], 512);
            h = Lb / nc[d];
            ih[d] = (float)(nc[d] / Lb);
        } else {
            double lo = 1e300, hi = -1e300;
            for (int i = 0; i < c->n; ++i) {
                lo = std::min(lo, q[3 * i + d]);
                hi = std::max(hi, q[3 * i + d]);
            }
            lo -= 5.0;
            hi += 5.0;
            const double ext = hi - lo;
            if (std::isfinite(edge_min)) {
                h = std::max(edge_min, ext / 256.0);
                nc[d] = std::max(1, (int)std::floor(ext / h));
                ih[d] = (float)(1.0 / h);
            }
            org[d] = (float)lo;
        }
        hh[d] = (float)h;
        m[d] = std::isfinite(reach) ? (int)std::ceil(reach / h) : 0;
    }
    const int ncell = nc[0] * nc[1] * nc[2];
    if (ncell > c->ncell_alloc) {
        int r;
        if ((r = dalloc(c, &s.cell_count, ncell)) || (r = dalloc(c, &s.cell_start, ncell + 1)) ||
            (r = dalloc(c, &s.cell_fill, ncell)))
            return r;
        c->ncell_alloc = ncell;
    }
    s.ncx = nc[0];
    s.ncy = nc[1];
    s.ncz = nc[2];
    s.ox = org[0];
    s.oy = org[1];
    s.oz = org[2];
    s.ihx = ih[0];
    s.ihy = ih[1];
    s.ihz = ih[2];
    s.hx = hh[0];
    s.hy = hh[1];
    s.hz = hh[2];
    s.mx = m[0];
    s.my = m[1];
    s.mz = m[2];
    c->pp.rcull = std::isfinite(reach) ? (float)(reach + 1e-3) : INFINITY;
    return BOUNCE_OK;
}

// Cluster-pair grid for the current host positions (finite cutoff, one
// system): columns of edge ~ (8 / density)^(1/3) over (x, y), so that a
// cluster of 8 z-sorted atoms is roughly a cube; capacities from the host
// positions with margins (an overflow during a run is reported as
// BOUNCE_ERR_LIST_OVERFLOW).  A droplet keeps its grid while every atom
// stays inside it, so that captured graphs stay valid.
// Largest prune skin of the cluster lists (A).
#ifndef CL_PRUNE_SKIN
#define CL_PRUNE_SKIN 0.8
#endif

int setup_clusters(bounce_ctx* c, const double* q) {
    DevClu& k = c->ds.cl;
    const bounce_config& g = c->cfg;
    const int n = c->n;
    if (!finite_cut(g) || c->ds.rep_of) {
        k.on = 0;
        return BOUNCE_OK;
    }
    const double cskin = g.pair_skin > 0 ? g.pair_skin : g.skin;
    const double rl = g.r_cut + cskin;
    const bool two = g.jump_coulomb && g.r_off < g.r_cut;
    const double rsh = std::min(g.r_off, g.r_cut) + cskin;
    double lo[3], hi[3];
    for (int d = 0; d < 3; ++d) {
        if (g.periodic) {
            lo[d] = 0.0;
            hi[d] = g.box[d];
        } else {
            lo[d] = 1e300;
            hi[d] = -1e300;
            for (int i = 0; i < n; ++i) {
                lo[d] = std::min(lo[d], q[3 * i + d]);
                hi[d] = std::max(hi[d], q[3 * i + d]);
            }
        }
    }
    // keep the current grid (a periodic box's is fixed; a droplet's while
    // every atom lies inside it) while the columns stay well inside capacity
    if (k.on && !c->cl_force) {
        const double x0 = k.ox, y0 = k.oy, x1 = k.ox + k.ncx / k.ihx, y1 = k.oy + k.ncy / k.ihy;
        if (g.periodic || (lo[0] >= x0 && lo[1] >= y0 && hi[0] <= x1 && hi[1] <= y1)) {
            std::vector<int> cnt(k.ncol, 0);
            int mx = 0;
            for (int i = 0; i < n; ++i) {
                double x = q[3 * i], y = q[3 * i + 1];
                if (g.periodic) {
                    x -= g.box[0] * std::floor(x / g.box[0]);
                    y -= g.box[1] * std::floor(y / g.box[1]);
                }
                const int cx = std::min(std::max((int)std::floor((x - x0) * k.ihx), 0), k.ncx - 1);
                const int cy = std::min(std::max((int)std::floor((y - y0) * k.ihy), 0), k.ncy - 1);
                mx = std::max(mx, ++cnt[cy * k.ncx + cx]);
            }
            if (4 * mx <= 3 * k.maxcol) return BOUNCE_OK;
        }
    }
    double vol = 1.0;
    for (int d = 0; d < 3; ++d) {
        if (!g.periodic) {
            lo[d] -= 2.0;
            hi[d] += 2.0;
        }
        vol *= hi[d] - lo[d];
    }
    // a droplet fills about half of its bounding box
    const double rho = std::max(n / (g.periodic ? vol : 0.55 * vol), 1e-4);
    double a = std::min(std::max(std::cbrt(8.0 / rho) * c->cl_edge_factor, 2.5), 12.0);
    c->cl_force = false;
    int nc[2];
    for (;;) {
        for (int d = 0; d < 2; ++d) nc[d] = std::max(1, (int)std::floor((hi[d] - lo[d]) / a));
        if ((long long)nc[0] * nc[1] <= 65536) break;
        a *= 1.25;
    }
    DevClu nk = k;
    nk.on = 1;
    nk.ncx = nc[0];
    nk.ncy = nc[1];
    nk.ncol = nc[0] * nc[1];
    nk.ox = g.periodic ? 0.f : (float)lo[0];
    nk.oy = g.periodic ? 0.f : (float)lo[1];
    nk.ihx = (float)(nc[0] / (hi[0] - lo[0]));
    nk.ihy = (float)(nc[1] / (hi[1] - lo[1]));
    std::vector<int> cnt(nk.ncol, 0);
    int mx = 0;
    for (int i = 0; i < n; ++i) {
        double x = q[3 * i], y = q[3 * i + 1];
        if (g.periodic) {
            x -= g.box[0] * std::floor(x / g.box[0]);
            y -= g.box[1] * std::floor(y / g.box[1]);
        }
        const int cx = std::min(std::max((int)std::floor((x - nk.ox) * nk.ihx), 0), nk.ncx - 1);
        const int cy = std::min(std::max((int)std::floor((y - nk.oy) * nk.ihy), 0), nk.ncy - 1);
        mx = std::max(mx, ++cnt[cy * nk.ncx + cx]);
    }
    const int want = (mx * 3 / 2 + 16 + 7) / 8 * 8;
    if (mx > BOUNCE_CL_MAXCOL) return fail(c, BOUNCE_ERR_UNSUPPORTED, "a cluster column holds more than 1024 atoms");
    nk.maxcol = std::min(want, BOUNCE_CL_MAXCOL);
    nk.maxcl = nk.maxcol / BOUNCE_CL;
    const int ncl = nk.ncol * nk.maxcl;
    // lists: atoms within the search radius R of a cluster box of edge ~a
    // (its volume by Steiner's formula), with a margin; the lower clusters of
    // the order hold up to the whole count, the mean is half of it
    const double rho_a = std::max(n / (g.periodic ? vol : 0.52 * vol), 0.02);
    const double rr[2] = {rl, rsh};
    nk.nlists = two ? 2 : 1;
    for (int L = 0; L < 2; ++L) {
        const double R = rr[L];
        const double V = a * a * a + 6.0 * a * a * R + 3.0 * M_PI * a * R * R + 4.18879 * R * R * R;
        const int est = (int)(rho_a * V);
        nk.capj[L] = L < nk.nlists ? (est * 2 + 128 + 31) / 32 * 32 : 1;
        const double rm = rr[L] + 1e-3;
        nk.rsx[L] = (float)rm;
        nk.rs2[L] = (float)(rm * rm);
    }
    nk.cskin_half2 = 0.25 * cskin * cskin;
    nk.capitems = ncl * (nk.capj[0] / BOUNCE_CL_EPW + 1);
    // pruned lists: entries within r + dp of some atom of I, dp = half the
    // cluster skin up to CL_PRUNE_SKIN (10 mA margin for the FP32 test),
    // pruned again when an atom has moved dp / 2 (1 mA margin)
    {
        const double dp = std::min(0.5 * cskin, (double)CL_PRUNE_SKIN);
        for (int L = 0; L < 2; ++L) {
            const double rp = rr[L] - cskin + dp + 0.01;
            nk.prs2[L] = (float)(rp * rp);
        }
        const double hp = 0.5 * dp - 0.001;
        nk.pdisp2 = (float)(hp * hp);
    }
    int r;
    if (!c->cl_atoms_alloc) {
        if ((r = dalloc(c, &nk.col_atoms, n)) || (r = dalloc(c, &nk.atom_col, n)) || (r = dalloc(c, &nk.a2s, n)) ||
            (r = dalloc(c, &nk.crefx, n)) || (r = dalloc(c, &nk.crefy, n)) || (r = dalloc(c, &nk.crefz, n)) ||
            (r = dalloc(c, &nk.cofx, n)) || (r = dalloc(c, &nk.cofy, n)) || (r = dalloc(c, &nk.cofz, n)) ||
            (r = dalloc(c, &nk.rebuild, 1)) || (r = dalloc(c, &nk.done_ctr, 4)) || (r = dalloc(c, &nk.prune, 1)) ||
            (r = dalloc(c, &nk.pnitems, 6)))
            return r;
        c->cl_atoms_alloc = true;
    }
    if (nk.ncol > c->cl_cap_ncol) {
        if ((r = dalloc(c, &nk.col_count, nk.ncol)) || (r = dalloc(c, &nk.col_start, nk.ncol + 1)) ||
            (r = dalloc(c, &nk.col_fill, nk.ncol)) || (r = dalloc(c, &nk.col_ncl, nk.ncol)))
            return r;
        c->cl_cap_ncol = nk.ncol;
    }
    if (ncl > c->cl_cap_ncl) {
        const size_t sl = (size_t)ncl * BOUNCE_CL;
        if ((r = dalloc(c, &nk.cl_atom, sl)) || (r = dalloc(c, &nk.sphi[0], sl)) || (r = dalloc(c, &nk.sphi[1], sl)) ||
            (r = dalloc(c, &nk.splo[0], sl)) || (r = dalloc(c, &nk.splo[1], sl)) || (r = dalloc(c, &nk.smol, sl)) ||
            (r = dalloc(c, &nk.bb_lo, ncl)) || (r = dalloc(c, &nk.bb_hi, ncl)) || (r = dalloc(c, &nk.lcnt[0], ncl)) ||
            (r = dalloc(c, &nk.lcnt[1], ncl)) || (r = dalloc(c, &nk.acc, 3 * sl)) || (r = dalloc(c, &nk.pref, sl)) ||
            (r = dalloc(c, &nk.pcnt[0], ncl)) || (r = dalloc(c, &nk.pcnt[1], ncl)))
            return r;
        c->cl_cap_ncl = ncl;
    }
    for (int L = 0; L < 2; ++L)
        if ((size_t)ncl * nk.capj[L] > c->cl_cap_lst[L]) {
            if ((r = dalloc(c, &nk.lst[L], (size_t)ncl * nk.capj[L])) ||
                (r = dalloc(c, &nk.plst[L], (size_t)ncl * nk.capj[L])))
                return r;
            c->cl_cap_lst[L] = (size_t)ncl * nk.capj[L];
        }
    if (nk.capitems > c->cl_cap_items) {
        if ((r = dalloc(c, &nk.pitems[0], nk.capitems)) || (r = dalloc(c, &nk.pitems[1], nk.capitems))) return r;
        c->cl_cap_items = nk.capitems;
    }
    prepare_cluster_pairs();
    k = nk;
    return BOUNCE_OK;
}

// All-pairs tiles (systems without a cutoff): the static items of the
// current replica layout for j-blocks of c->tile_j atoms.
int setup_tiles(bounce_ctx* c) {
    DevTile& T = c->ds.tl;
    if (finite_cut(c->cfg)) {
        T.on = 0;
        return BOUNCE_OK;
    }
    if (c->rep_bounds.size() < 2) c->rep_bounds = {0, c->n};
    std::vector<int4> items;
    for (size_t r = 0; r + 1 < c->rep_bounds.size(); ++r) {
        const int b = c->rep_bounds[r], e = c->rep_bounds[r + 1];
        for (int i0 = b; i0 < e; i0 += 32)
            for (int j0 = i0; j0 < e; j0 += c->tile_j)
                items.push_back(make_int4(i0, std::min(32, e - i0), j0, std::min(c->tile_j, e - j0)));
    }
    int r;
    if ((int)items.size() > c->tile_cap) {
        if ((r = dalloc(c, &c->tile_items, items.size()))) return r;
        c->tile_cap = (int)items.size();
    }
    if (!T.acc && (r = dalloc(c, &T.acc, 3 * (size_t)c->n))) return r;
    CU(cudaMemcpy(c->tile_items, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice));
    T.on = 1;
    T.items = c->tile_items;
    T.nitems = (int)items.size();
    T.tj = c->tile_j;
    T.blocks = c->tile_blocks;
    drop_graphs(c);
    return BOUNCE_OK;
}

// Raise the cluster rebuild flag (positions were replaced).
int flag_clusters(bounce_ctx* c, cudaStream_t st) {
    if (!c->ds.cl.on) return BOUNCE_OK;
    static const int one = 1;
    CU(cudaMemcpyAsync(c->ds.cl.rebuild, &one, sizeof(int), cudaMemcpyHostToDevice, st));
    return BOUNCE_OK;
}

// Partners a jump can draw.  With LJ alone on the jumps (Coulomb wholly in
// F_0) and one bound per type, an atom of type a proposes only if L*_a > 0,
// and only the types b with LJ parameters for (a, b) interact with it
// through the jump part (the partner J is drawn among the particles
// interacting with i, Sec. V).  When that leaves out some present type, the
// jump rows keep only those partners (Params::jpart) and follow the
// displacement of the types that propose or are drawn.
void set_rows_kind(bounce_ctx* c, int kind);

void set_jump_partners(bounce_ctx* c, const std::vector<double>& sg, const std::vector<double>& ep) {
    const int T = c->n_types;
    bool present[BOUNCE_MAXT] = {};
    for (int i = 0; i < c->n; ++i) present[c->type[i]] = true;
    unsigned cells = 0, owners = 0;
    bool drops = false;
    for (int a = 0; a < BOUNCE_MAXT; ++a) {
        int m = 0;
        const bool owner = a < T && present[a] && c->Lstar[a] > 0.0;
        for (int b = 0; owner && b < T; ++b) {
            const bool lj = sg[a * T + b] != 0.0 && ep[a * T + b] != 0.0;
            if (lj) m |= 1 << b;
            else if (present[b]) drops = true;
        }
        c->pp.jpart[a] = m;
        cells |= (unsigned)m;
        if (owner) owners |= 1u << a;
    }
    c->pp.jcells = (int)cells;
    c->jfilter = !c->cfg.jump_coulomb && !c->cfg.pair_bounds && drops;
    c->jmove = owners | cells;
    set_rows_kind(c, 0);
}

// Launch the rebuild sequence of the candidate rows (gated by the device
// flag unless forced).  After BAOAB runs on clusters the step kernel did not
// test the rows' displacement, so it is tested here first, at the current
// positions (the test the oracle applies before every use of the rows).
void rebuild(bounce_ctx* c, int step_off, bool force, cudaStream_t st, int mode = ROWS_ALL) {
    if (c->rows_check_due) {
        long long step = c->cur_step;
        if (step_off == 0) launch_flag_moved(c->ds, c->pp, (int)(step & 1), st);
        c->rows_check_due = false;
    }
    launch_rebuild(c->ds, c->pp, step_off, force, c->bitmap_warps, c->bitmap_bytes, mode, st);
}

// Row-build mode of the runs of `integ`: the jump step is the rows' only
// reader when the pair sums run over clusters or tiles (and no short rows
// exist), so atoms of a type with L* = 0 need none.
int rows_mode(const bounce_ctx* c, int integ) {
    if (integ == BOUNCE_BAOAB || c->ds.rep_of || !(c->ds.cl.on || c->ds.tl.on) || c->pp.rshort2 < INFINITY ||
        !c->ds.act_order)
        return ROWS_ALL;
    for (int a = 0; a < c->pp.n_types; ++a)
        if (c->Lstar[a] == 0.0) return ROWS_ACTIVE;
    return ROWS_ALL;
}

// Entry points that read every row (energies, histograms, gradients over
// the rows, the rows themselves) first build the rows a run left empty, at
// the current positions; the displacement test of the rows keeps the
// reference positions of the last full build, so the next run's rebuilds
// come at the same steps as without this call.
void complete_rows(bounce_ctx* c, cudaStream_t st) {
    if (!c->rows_partial) return;
    launch_rebuild(c->ds, c->pp, 0, true, c->bitmap_warps, c->bitmap_bytes, ROWS_IDLE, st);
    c->rows_partial = false;
}

// Whether the runs of `integ` read jump rows that keep only the partners a
// jump can draw (the jump step is then the rows' only reader).
bool jump_filtered(const bounce_ctx* c, int integ) {
    return c->jfilter && integ != BOUNCE_BAOAB && (c->ds.cl.on || c->ds.tl.on || c->ds.rep_of) &&
           !(c->pp.rshort2 < INFINITY);
}

// Row-build mode of the gated rebuilds inside the runs of `integ`.
int run_rows_mode(const bounce_ctx* c, int integ) {
    return rows_mode(c, integ) | (jump_filtered(c, integ) ? ROWS_FILTER : 0);
}

// What the rows buffers hold (0 nothing usable, 1 full rows, 2 jump rows);
// the displacement test follows the types that can change them.
void set_rows_kind(bounce_ctx* c, int kind) {
    c->rows_kind = kind;
    c->ds.rows_move = kind == 2 ? c->jmove : ~0u;
}

// Exchange the run's row buffers and the readers' ones.
void swap_rows(bounce_ctx* c) {
    if (!c->rows_swapped) {
        c->rows_main = c->ds.rows;
        c->nlong_main = c->ds.nlong;
        c->ds.rows = c->rows_alt;
        c->ds.nlong = c->nlong_alt;
    } else {
        c->ds.rows = c->rows_main;
        c->ds.nlong = c->nlong_main;
    }
    c->rows_swapped = !c->rows_swapped;
}

// Rows for the entry points that read every row (energies, histograms,
// gradients, the rows themselves, the pair forward, the stand-alone jump
// half-step); `replaced`: the positions were just set.  With jump rows that
// keep only the jump partners, the full rows are built at the current
// positions into the readers' buffers, so that the run's rows, their
// reference positions and the rebuild flag stay as the last run left them.
int prepare_readers(bounce_ctx* c, cudaStream_t st, bool replaced = false) {
    if (!c->jfilter) {
        rebuild(c, 0, replaced, st);
        complete_rows(c, st);
        return BOUNCE_OK;
    }
    if (replaced) {
        ++c->pos_version;
        set_rows_kind(c, 0);  // the next run builds its rows afresh
    }
    if (c->rows_swapped && c->reader_version == c->pos_version) return BOUNCE_OK;
    if (!c->rows_alt) {
        int r;
        if ((r = dalloc(c, &c->rows_alt, (size_t)c->n * c->ds.cap)) || (r = dalloc(c, &c->nlong_alt, c->n)))
            return r;
    }
    if (!c->rows_swapped) swap_rows(c);
    launch_rebuild(c->ds, c->pp, 0, true, c->bitmap_warps, c->bitmap_bytes, ROWS_READER, st);
    c->reader_version = c->pos_version;
    return BOUNCE_OK;
}

int check_err(bounce_ctx* c, cudaStream_t st) {
    CU(cudaMemcpyAsync(c->h_err, c->ds.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    if (*c->h_err & BERR_RATE) {
        cudaMemsetAsync(c->ds.err, 0, sizeof(int), st);
        return fail(c, BOUNCE_ERR_NONFINITE, "a jump proposal mean was not finite or above 1e6 (the state blew up)");
    }
    if (*c->h_err & (BERR_LIST_OVERFLOW | BERR_SHORT_OVERFLOW)) {
        const int e = *c->h_err;
        cudaMemsetAsync(c->ds.err, 0, sizeof(int), st);
        return fail(c, BOUNCE_ERR_LIST_OVERFLOW,
                    (e & BERR_LIST_OVERFLOW) ? "a candidate row exceeded max_neighbors"
                                             : "a short-range row exceeded max_short");
    }
    return BOUNCE_OK;
}

// What happens at one step boundary: whether the reciprocal gradient is
// evaluated there and the time hr it kicks over (see k_step).
void plan(const bounce_ctx* c, int integ, int variant, long long step, bool& pme, double& hr, double& hout) {
    const double dt = c->cfg.dt_fs;
    const double hk = variant == 1 ? dt : 0.5 * dt;
    pme = false;
    hr = 0.0;
    hout = 0.0;
    if (integ == BOUNCE_BOUNCE_RESPA || integ == BOUNCE_BOUNCE_RESPA_EXT) {
        const int m = c->cfg.respa_m;
        if (step % m == 0) {
            const double H = (variant == 1 ? 1.0 : 0.5) * m * dt;
            pme = c->has_pme;
            hr = c->has_pme ? H : 0.0;
            if (integ == BOUNCE_BOUNCE_RESPA_EXT) hout = H;
        }
        return;
    }
    if (integ == BOUNCE_BOUNCE_RESPA1) {
        // kicks that meet at one boundary act at the same positions: the
        // short-range kick of the intermediate level and the reciprocal kick
        // of the outer level are applied together
        const int m = c->cfg.respa_m, m2 = c->cfg.respa_m2;
        const double w = variant == 1 ? 1.0 : 0.5;
        if (step % m == 0) hout = w * m * dt;
        if (step % ((long long)m * m2) == 0 && c->has_pme) {
            pme = true;
            hr = w * m * m2 * dt;
        }
        return;
    }
    if (c->has_pme) {
        pme = true;
        hr = hk;
    }
}

// System view of a run of `integ`: BAOAB on clusters needs no candidate
// rows, so its step kernel does not test them (rows_flag = 0).
DevSys run_view(const bounce_ctx* c, int integ) {
    DevSys s = c->ds;
    s.rows_flag = (integ == BOUNCE_BAOAB && s.cl.on) ? 0 : 1;
    const int sk = c->cfg.step_kernel;
    s.lite = sk == 2 ? 1 : (sk == 1 ? 0 : ((integ == BOUNCE_BAOAB || c->lite_jumps) ? 1 : 0));
    return s;
}

// Expected jump proposals per atom-step from the bounds: beta <|v_a|> L*_a
// n delta summed over the atoms' types, with <|v_a|> = sqrt(8 k_B T / (pi
// m_a)) and n the atoms within r_list at density rho (an upper bound of the
// rate: the per-type-pair bounds only lower it).
double expected_proposals(const bounce_ctx* c, double rho) {
    const bounce_config& g = c->cfg;
    const double beta = 1.0 / (KB_D * g.temperature_K);
    const double rl = r_list(g);
    const double nbar = std::isfinite(rl) ? std::min((double)c->n, rho * 4.18879 * rl * rl * rl) : (double)c->n;
    // jump rows that keep only the jump partners: the share of the atoms of a partner type
    double share[BOUNCE_MAXT];
    for (int a = 0; a < BOUNCE_MAXT; ++a) {
        int k = 0;
        if (c->jfilter)
            for (int i = 0; i < c->n; ++i) k += (c->pp.jpart[a] >> c->type[i]) & 1;
        share[a] = c->jfilter && c->n ? (double)k / c->n : 1.0;
    }
    double sum = 0.0;
    for (int i = 0; i < c->n; ++i) {
        const double vbar = std::sqrt(8.0 * KB_D * g.temperature_K * ACCEL_D / (M_PI * c->mass[i]));
        sum += beta * vbar * c->Lstar[c->type[i]] * nbar * share[c->type[i]] * g.dt_fs;
    }
    return sum / c->n;
}

// The gated rebuilds at one step boundary: the clusters (their own flag) and
// the candidate rows, which only the jump step reads (BOUNCE integrators, or
// every integrator without clusters, whose pair sums run over the rows).
void rebuild_for(bounce_ctx* c, int integ, int off, cudaStream_t st) {
    if (c->ds.cl.on) launch_cluster_rebuild(c->ds, c->pp, off, false, st);
    if (!c->ds.cl.on || integ != BOUNCE_BAOAB) rebuild(c, off, false, st, run_rows_mode(c, integ));
}

// Before a run: rows a previous run left partial are completed when this
// run builds full rows; after it, they are partial if it built active ones.
// With jump rows that keep only the jump partners, the run's buffers come
// back from the readers, and rows of the other kind (full rows for a run
// that reads them, jump rows for a BOUNCE run) are rebuilt at once.
void rows_before_run(bounce_ctx* c, int integ, cudaStream_t st) {
    if (c->rows_swapped) swap_rows(c);
    if (!c->jfilter) {
        if (rows_mode(c, integ) == ROWS_ALL) complete_rows(c, st);
        return;
    }
    if (c->ds.cl.on && integ == BOUNCE_BAOAB) return;  // reads no rows
    const int kind = jump_filtered(c, integ) ? 2 : 1;
    if (c->rows_kind != kind) {
        set_rows_kind(c, kind);
        rebuild(c, 0, true, st, kind == 2 ? run_rows_mode(c, integ) : ROWS_ALL);
        c->rows_partial = false;
    }
}
void rows_after_run(bounce_ctx* c, int integ) {
    ++c->pos_version;
    if (rows_mode(c, integ) == ROWS_ACTIVE) c->rows_partial = true;
}

void boundary(bounce_ctx* c, int integ, int variant, int off, long long step, cudaStream_t st) {
    bool pme;
    double hr, hout;
    plan(c, integ, variant, step, pme, hr, hout);
    rebuild_for(c, integ, off, st);
    if (pme) launch_pme(c->ds, c->pp, c->pme, off, st);
    launch_step(run_view(c, integ), c->pp, integ, variant, off, hr, hout, st);
}

// Steps after which the kick pattern of the integrator repeats.
int respa_period(const bounce_ctx* c, int integ) {
    if (integ == BOUNCE_BOUNCE_RESPA || integ == BOUNCE_BOUNCE_RESPA_EXT) return c->cfg.respa_m;
    if (integ == BOUNCE_BOUNCE_RESPA1) return c->cfg.respa_m * c->cfg.respa_m2;
    return 1;
}

// Graph of CHUNK body steps whose first step index is congruent to `phase`
// modulo the integrator's period (the RESPA block boundaries inside a chunk
// depend on it).
int ensure_graph(bounce_ctx* c, int integ, int phase) {
    if (c->graph[integ][phase]) return BOUNCE_OK;
    cudaStream_t st = c->cap_stream;
    cudaGraph_t g = nullptr;
    CU(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    for (int k = 0; k < CHUNK; ++k) boundary(c, integ, 1, k, (long long)phase + k, st);
    launch_advance_step(c->ds, CHUNK, st);
    CU(cudaStreamEndCapture(st, &g));
    cudaError_t e = cudaGraphInstantiate(&c->graph[integ][phase], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(c, BOUNCE_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    return BOUNCE_OK;
}

int check_run_args(bounce_ctx* c, int64_t n_steps, int32_t integ) {
    if (n_steps < 0 || integ < BOUNCE_BAOAB || integ > BOUNCE_BOUNCE_RESPA1)
        return fail(c, BOUNCE_ERR_INVALID_ARG, "bad run arguments");
    if (integ == BOUNCE_BOUNCE_RESPA1) {
        const long long P = (long long)c->cfg.respa_m * c->cfg.respa_m2;
        if (n_steps % P != 0 || c->cur_step % P != 0)
            return fail(c, BOUNCE_ERR_INVALID_ARG, "BOUNCE-RESPA1 runs whole outer steps (multiples of respa_m respa_m2)");
    }
    if (integ == BOUNCE_BOUNCE_RESPA || integ == BOUNCE_BOUNCE_RESPA_EXT) {
        const int m = c->cfg.respa_m;
        if (integ == BOUNCE_BOUNCE_RESPA && !c->has_pme)
            return fail(c, BOUNCE_ERR_INVALID_ARG, "BOUNCE-RESPA needs an SPME grid");
        if (n_steps % m != 0 || c->cur_step % m != 0)
            return fail(c, BOUNCE_ERR_INVALID_ARG, "BOUNCE-RESPA runs whole outer steps (multiples of respa_m)");
    }
    return BOUNCE_OK;
}

}  // namespace

extern "C" {

void bounce_config_default(bounce_config* cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->dt_fs = 1.0;
    cfg->gamma_per_fs = 0.001;
    cfg->temperature_K = 300.0;
    cfg->seed = 0;
    cfg->r_on = 4.0;
    cfg->r_off = 5.0;
    cfg->r_cut = INFINITY;
    cfg->skin = 1.0;
    cfg->ewald_beta = 0.0;
    cfg->periodic = 0;
    cfg->max_neighbors = 2048;
    cfg->max_short = 256;
    cfg->device = 0;
    cfg->pme_order = 5;
    cfg->respa_m = 2;
    cfg->jump_coulomb = 1;
    cfg->respa_m2 = 3;
}

int bounce_create(bounce_ctx** out, const bounce_config* cfg) {
    bounce_ctx* c = nullptr;
    if (!out || !cfg) return BOUNCE_ERR_INVALID_ARG;
    *out = nullptr;
    if (!(cfg->dt_fs > 0) || !(cfg->temperature_K > 0) || cfg->gamma_per_fs < 0 || cfg->skin < 0 ||
        cfg->max_neighbors < 1 || cfg->max_short < 1 || !(cfg->r_off >= cfg->r_on) || cfg->r_on < 0 ||
        cfg->ewald_beta < 0 || !(cfg->pair_skin >= 0) || cfg->step_kernel < 0 || cfg->step_kernel > 2)
        return BOUNCE_ERR_INVALID_ARG;
    if (cfg->periodic && !(cfg->box[0] > 0 && cfg->box[1] > 0 && cfg->box[2] > 0)) return BOUNCE_ERR_INVALID_ARG;
    if (cfg->respa_m < 1 || cfg->respa_m > 8 || cfg->respa_m2 < 1 || cfg->respa_m2 > 8) return BOUNCE_ERR_INVALID_ARG;
    // two-stage choice: the row weight n_i * 65537 must fit 32 bits
    if (cfg->pair_bounds && cfg->max_neighbors >= 65535) return BOUNCE_ERR_UNSUPPORTED;
    c = new bounce_ctx();
    c->cfg = *cfg;
    cudaError_t e = cudaSetDevice(cfg->device);
    if (e != cudaSuccess) {
        delete c;
        return BOUNCE_ERR_CUDA;
    }
    if (cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMallocHost(&c->h_err, sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&c->h_cnt, CNT_N * sizeof(unsigned long long)) != cudaSuccess) {
        delete c;
        return BOUNCE_ERR_CUDA;
    }
    *out = c;
    return BOUNCE_OK;
}

int bounce_set_topology(bounce_ctx* c, int32_t n, const int32_t* type, const double* mass, const double* charge,
                        const int32_t* molecule, int32_t nb, const int32_t* bond_ij, const double* bond_k_r0,
                        int32_t na, const int32_t* angle_ijk, const double* angle_k_t0) {
    if (!c) return BOUNCE_ERR_INVALID_ARG;
    if (n < 1 || !type || !mass || !charge || !molecule || nb < 0 || na < 0 || (nb && (!bond_ij || !bond_k_r0)) ||
        (na && (!angle_ijk || !angle_k_t0)))
        return fail(c, BOUNCE_ERR_INVALID_ARG, "bad topology arguments");
    cudaSetDevice(c->cfg.device);
    free_all(c);
    c->ncell_alloc = 0;
    c->have_topo = c->have_lj = c->have_state = false;
    c->rows_valid = false;
    c->n = n;
    c->type.assign(type, type + n);
    c->mol.assign(molecule, molecule + n);
    c->mass.assign(mass, mass + n);
    c->charge.assign(charge, charge + n);
    int maxt = 0;
    for (int i = 0; i < n; ++i) {
        if (type[i] < 0 || type[i] >= BOUNCE_MAXT) return fail(c, BOUNCE_ERR_INVALID_ARG, "atom type out of range");
        if (!(mass[i] > 0) || !std::isfinite(charge[i])) return fail(c, BOUNCE_ERR_INVALID_ARG, "bad mass or charge");
        maxt = std::max(maxt, type[i] + 1);
    }
    c->n_types = maxt;
    // bonded terms per atom
    std::vector<std::vector<std::pair<int4, float2>>> per(n);
    for (int b = 0; b < nb; ++b) {
        int i = bond_ij[2 * b], j = bond_ij[2 * b + 1];
        if (i < 0 || j < 0 || i >= n || j >= n || i == j) return fail(c, BOUNCE_ERR_INVALID_ARG, "bad bond");
        float2 kp = make_float2((float)bond_k_r0[2 * b], (float)bond_k_r0[2 * b + 1]);
        per[i].push_back({make_int4(0, j, 0, 0), kp});
        per[j].push_back({make_int4(0, i, 0, 0), kp});
    }
    for (int a = 0; a < na; ++a) {
        int i = angle_ijk[3 * a], v = angle_ijk[3 * a + 1], k = angle_ijk[3 * a + 2];
        if (i < 0 || v < 0 || k < 0 || i >= n || v >= n || k >= n || i == v || v == k || i == k)
            return fail(c, BOUNCE_ERR_INVALID_ARG, "bad angle");
        float2 kp = make_float2((float)angle_k_t0[2 * a], (float)angle_k_t0[2 * a + 1]);
        per[i].push_back({make_int4(1, v, k, 0), kp});
        per[k].push_back({make_int4(1, v, i, 0), kp});
        per[v].push_back({make_int4(2, i, k, 0), kp});
    }
    c->bt_off.assign(n + 1, 0);
    c->bt_idx.clear();
    c->bt_par.clear();
    for (int i = 0; i < n; ++i) {
        c->bt_off[i + 1] = c->bt_off[i] + (int)per[i].size();
        for (auto& t : per[i]) {
            c->bt_idx.push_back(t.first);
            c->bt_par.push_back(t.second);
        }
    }
    // device buffers
    DevSys& s = c->ds;
    s.n = n;
    int r;
    for (int b = 0; b < 2; ++b) {
        if ((r = dalloc(c, &s.qx[b], n)) || (r = dalloc(c, &s.qy[b], n)) || (r = dalloc(c, &s.qz[b], n)) ||
            (r = dalloc(c, &s.phi[b], n)) || (r = dalloc(c, &s.plo[b], n)))
            return r;
    }
    double *kick, *osd;
    int *dtype, *dmol, *boff;
    int4* bidx;
    float2* bpar;
    const double rl = r_list(c->cfg);
    s.cap = std::isfinite(rl) ? c->cfg.max_neighbors : std::max(1, std::min(n - 1, c->cfg.max_neighbors));
    const double rs = c->cfg.r_off + c->cfg.skin;
    // Short rows exist only when they are a strict subset of the long rows;
    // otherwise F_0 reads the long rows (rshort2 = +inf) and one slot is kept.
    const bool distinct_short = short_rows(c->cfg) && rs < rl;
    s.caps = distinct_short ? c->cfg.max_short : 1;
    if ((r = dalloc(c, &s.vx, n)) || (r = dalloc(c, &s.vy, n)) || (r = dalloc(c, &s.vz, n)) ||
        (r = dalloc(c, &kick, n)) || (r = dalloc(c, &osd, n)) || (r = dalloc(c, &dtype, n)) ||
        (r = dalloc(c, &dmol, n)) || (r = dalloc(c, &boff, n + 1)) ||
        (r = dalloc(c, &bidx, c->bt_idx.size())) || (r = dalloc(c, &bpar, c->bt_par.size())) ||
        (r = dalloc(c, &s.nlong, n)) || (r = dalloc(c, &s.rows, (size_t)n * s.cap)) ||
        (r = dalloc(c, &s.nseg, (size_t)n * BOUNCE_MAXT)) || (r = dalloc(c, &s.nshort, n)) || (r = dalloc(c, &s.srows, distinct_short ? (size_t)n * s.caps : 1)) ||
        (r = dalloc(c, &s.refx, n)) || (r = dalloc(c, &s.refy, n)) || (r = dalloc(c, &s.refz, n)) ||
        (r = dalloc(c, &s.cell_atoms, n)) || (r = dalloc(c, &s.cell_phi, n)) || (r = dalloc(c, &s.cell_mol, n)) ||
        (r = dalloc(c, &s.g0, n)) ||
        (r = dalloc(c, &s.cell_type, n)) ||
        (r = dalloc(c, &s.done_ctr, 2)) ||
        (r = dalloc(c, &s.rebuild, 1)) || (r = dalloc(c, &s.err, 1)) ||
        (r = dalloc(c, &s.cnt, CNT_N)) || (r = dalloc(c, &c->d_step, 1)) || (r = dalloc(c, &c->terms, 6 * (size_t)n + 2048)) ||
        (r = dalloc(c, &c->d_stage, 6 * (size_t)n)))
        return r;
    s.kick = kick;
    s.osd = osd;
    s.type = dtype;
    s.mol = dmol;
    s.bt_off = boff;
    s.bt_idx = bidx;
    s.bt_par = bpar;
    s.step_base = c->d_step;
    s.rows_flag = 1;
    s.rows_move = ~0u;
    std::vector<double> hk(n), ho(n);
    const double c1 = std::exp(-c->cfg.gamma_per_fs * c->cfg.dt_fs);
    for (int i = 0; i < n; ++i) {
        hk[i] = ACCEL_D / mass[i];
        ho[i] = std::sqrt((1.0 - c1 * c1) * KB_D * c->cfg.temperature_K * ACCEL_D / mass[i]);
    }
    CU(cudaMemcpy(kick, hk.data(), n * sizeof(double), cudaMemcpyHostToDevice));
    CU(cudaMemcpy(osd, ho.data(), n * sizeof(double), cudaMemcpyHostToDevice));
    CU(cudaMemcpy(dtype, type, n * sizeof(int), cudaMemcpyHostToDevice));
    CU(cudaMemcpy(dmol, molecule, n * sizeof(int), cudaMemcpyHostToDevice));
    CU(cudaMemcpy(boff, c->bt_off.data(), (n + 1) * sizeof(int), cudaMemcpyHostToDevice));
    if (!c->bt_idx.empty()) {
        CU(cudaMemcpy(bidx, c->bt_idx.data(), c->bt_idx.size() * sizeof(int4), cudaMemcpyHostToDevice));
        CU(cudaMemcpy(bpar, c->bt_par.data(), c->bt_par.size() * sizeof(float2), cudaMemcpyHostToDevice));
    }
    // charge and type ride in the w slots of the split positions
    std::vector<float4> hh(n), hl(n);
    for (int i = 0; i < n; ++i) {
        int t = type[i];
        float tf;
        std::memcpy(&tf, &t, 4);
        hh[i] = make_float4(0.f, 0.f, 0.f, (float)charge[i]);
        hl[i] = make_float4(0.f, 0.f, 0.f, tf);
    }
    for (int b = 0; b < 2; ++b) {
        CU(cudaMemcpy(s.phi[b], hh.data(), n * sizeof(float4), cudaMemcpyHostToDevice));
        CU(cudaMemcpy(s.plo[b], hl.data(), n * sizeof(float4), cudaMemcpyHostToDevice));
    }
    // Row builder: per warp, the bitmaps over a window of atom indices (one
    // per partner type with per-type-pair bounds, plus the short-row bitmap
    // when short rows exist) and 3 x 128 ints of cell-row runs, at most 8 KB;
    // the window spans every atom when that fits (short rows need it).
    const int words = (n + 31) / 32;
    const int nbm = (c->cfg.pair_bounds ? c->n_types : 1) + (distinct_short ? 1 : 0);
    const int wmax = ((8192 - 3 * 128 * 4) / (4 * nbm)) & ~3;
    c->bitmap_warps = std::min((words + 3) & ~3, wmax);  // window words per bitmap
    c->bitmap_bytes = (size_t)8 * ((size_t)nbm * c->bitmap_warps + 3 * 128) * 4;
    nlist_set_smem_limit(c->bitmap_bytes);
    c->rep_bounds = {0, n};
    if ((r = setup_tiles(c))) return r;
    c->have_topo = true;
    return BOUNCE_OK;
}

int bounce_set_lj(bounce_ctx* c, int32_t T, const double* sigma, const double* eps) {
    if (!c) return BOUNCE_ERR_INVALID_ARG;
    if (!c->have_topo) return fail(c, BOUNCE_ERR_STATE, "set the topology first");
    if (T < c->n_types || T > BOUNCE_MAXT || !sigma || !eps) return fail(c, BOUNCE_ERR_INVALID_ARG, "bad LJ table");
    std::vector<double> sg(c->n_types * c->n_types), ep(c->n_types * c->n_types);
    for (int a = 0; a < c->n_types; ++a)
        for (int b = 0; b < c->n_types; ++b) {
            sg[a * c->n_types + b] = sigma[a * T + b];
            ep[a * c->n_types + b] = eps[a * T + b];
        }
    compute_bounds(c, sg, ep);
    fill_params(c, sg, ep);
    set_jump_partners(c, sg, ep);
    drop_graphs(c);
    {
        // atoms that can propose (L* > 0) first, for the row builder
        std::vector<int> order;
        order.reserve(c->n);
        for (int pass = 0; pass < 2; ++pass)
            for (int i = 0; i < c->n; ++i)
                if ((c->Lstar[c->type[i]] > 0.0) == (pass == 0)) order.push_back(i);
        int nact = 0;
        for (int i = 0; i < c->n; ++i) nact += c->Lstar[c->type[i]] > 0.0 ? 1 : 0;
        if (!c->d_act_order) {
            int r = dalloc(c, &c->d_act_order, c->n);
            if (r) return r;
        }
        CU(cudaMemcpy(c->d_act_order, order.data(), c->n * sizeof(int), cudaMemcpyHostToDevice));
        c->ds.act_order = c->d_act_order;
        c->ds.n_act = nact;
    }
    if (!c->has_pme) {
        int r = setup_pme(c);
        if (r) return r;
    }
    c->have_lj = true;
    return BOUNCE_OK;
}

int bounce_set_state(bounce_ctx* c, const double* q, const double* v, int64_t step, int32_t where, void* stream) {
    if (!c) return BOUNCE_ERR_INVALID_ARG;
    if (!c->have_topo || !c->have_lj) return fail(c, BOUNCE_ERR_STATE, "set the topology and LJ table first");
    if (!q || !v || (where != BOUNCE_HOST && where != BOUNCE_DEVICE) || step < 0)
        return fail(c, BOUNCE_ERR_INVALID_ARG, "bad state arguments");
    cudaSetDevice(c->cfg.device);
    cudaStream_t st = (cudaStream_t)stream;
    const int n = c->n;
    const size_t n3 = 3 * (size_t)n;
    if (!c->h_stage) CU(cudaMallocHost(&c->h_stage, 2 * n3 * sizeof(double)));
    // host view of the state for the checks and the cell grid
    const double *hq = q, *hv = v;
    if (where == BOUNCE_DEVICE) {
        CU(cudaMemcpyAsync(c->h_stage, q, n3 * sizeof(double), cudaMemcpyDeviceToHost, st));
        CU(cudaMemcpyAsync(c->h_stage + n3, v, n3 * sizeof(double), cudaMemcpyDeviceToHost, st));
        CU(cudaStreamSynchronize(st));
        hq = c->h_stage;
        hv = c->h_stage + n3;
    }
    for (size_t k = 0; k < n3; ++k)
        if (!std::isfinite(hq[k]) || !std::isfinite(hv[k]))
            return fail(c, BOUNCE_ERR_NONFINITE, "non-finite position or velocity");
    // short rows (systems without a cutoff) need one row-builder window over every atom
    if (!c->ds.rep_of && c->pp.rshort2 < INFINITY && c->bitmap_warps < (c->n + 31) / 32)
        return fail(c, BOUNCE_ERR_UNSUPPORTED, "too many atoms for short rows without a cutoff");
    const DevSys before = c->ds;
    int r = setup_grid(c, hq);
    if (r) return r;
    if ((r = setup_clusters(c, hq))) return r;
    {
        // density for the rate estimate: the box, or half the droplet's bounding box
        double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300}, vol = 1.0;
        for (int i = 0; i < c->n; ++i)
            for (int d = 0; d < 3; ++d) {
                lo[d] = std::min(lo[d], hq[3 * i + d]);
                hi[d] = std::max(hi[d], hq[3 * i + d]);
            }
        for (int d = 0; d < 3; ++d) vol *= c->cfg.periodic ? c->cfg.box[d] : std::max(hi[d] - lo[d], 1.0);
        const double rho = c->n / (c->cfg.periodic ? vol : 0.55 * vol);
        const bool lite = expected_proposals(c, rho) < 0.5;
        if (lite != c->lite_jumps) drop_graphs(c);
        c->lite_jumps = lite;
    }
    // captured graphs hold the system view by value: recapture only if the grid changed
    const DevSys& g = c->ds;
    if (g.ncx != before.ncx || g.ncy != before.ncy || g.ncz != before.ncz || g.ox != before.ox || g.oy != before.oy ||
        g.oz != before.oz || g.ihx != before.ihx || g.ihy != before.ihy || g.ihz != before.ihz ||
        g.mx != before.mx || g.my != before.my || g.mz != before.mz ||
        g.cell_count != before.cell_count || g.cell_start != before.cell_start || g.cell_fill != before.cell_fill ||
        std::memcmp(&g.cl, &before.cl, sizeof(DevClu)) != 0)
        drop_graphs(c);
    const int cur = (int)(step & 1);
    DevSys& s = c->ds;
    // host arrays: one pinned staging copy and one contiguous upload; device
    // arrays are read in place
    const double *dq = q, *dv = v;
    if (where == BOUNCE_HOST) {
        std::memcpy(c->h_stage, q, n3 * sizeof(double));
        std::memcpy(c->h_stage + n3, v, n3 * sizeof(double));
        CU(cudaMemcpyAsync(c->d_stage, c->h_stage, 2 * n3 * sizeof(double), cudaMemcpyHostToDevice, st));
        dq = c->d_stage;
        dv = c->d_stage + n3;
    }
    launch_state_in(s, dq, dv, cur, st);
    long long st0 = step;
    CU(cudaMemcpyAsync(c->d_step, &st0, sizeof(long long), cudaMemcpyHostToDevice, st));
    launch_pack_positions(s, c->pp, cur, st);
    // rows stay valid while every atom is within skin/2 of where they were
    // built (the same test as during a run); otherwise the next launch
    // rebuilds them
    if (c->rows_valid) {
        launch_flag_moved(s, c->pp, cur, st);
    } else {
        const int one = 1;
        CU(cudaMemcpyAsync(s.rebuild, &one, sizeof(int), cudaMemcpyHostToDevice, st));
        c->rows_valid = true;
    }
    if ((r = flag_clusters(c, st))) return r;
    c->rows_check_due = false;
    CU(cudaMemsetAsync(s.err, 0, sizeof(int), st));
    CU(cudaStreamSynchronize(st));
    c->step0 = step;
    c->cur_step = step;
    c->have_state = true;
    ++c->pos_version;
    return BOUNCE_OK;
}

int bounce_get_state(bounce_ctx* c, double* q, double* v, int32_t where, void* stream) {
    if (!c) return BOUNCE_ERR_INVALID_ARG;
    if (!c->have_state) return fail(c, BOUNCE_ERR_STATE, "no state");
    if (where != BOUNCE_HOST && where != BOUNCE_DEVICE) return fail(c, BOUNCE_ERR_INVALID_ARG, "bad where");
    cudaSetDevice(c->cfg.device);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t n3 = 3 * (size_t)c->n;
    if (where == BOUNCE_DEVICE) {
        // interleaved straight into the caller's device arrays, stream-ordered
        launch_state_out(c->ds, q, v, st);
        CU(cudaGetLastError());
        return BOUNCE_OK;
    }
    if (!c->h_stage) CU(cudaMallocHost(&c->h_stage, 2 * n3 * sizeof(double)));
    launch_state_out(c->ds, q ? c->d_stage : nullptr, v ? c->d_stage + n3 : nullptr, st);
    if (q) CU(cudaMemcpyAsync(c->h_stage, c->d_stage, n3 * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (v) CU(cudaMemcpyAsync(c->h_stage + n3, c->d_stage + n3, n3 * sizeof(double), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    if (q) std::memcpy(q, c->h_stage, n3 * sizeof(double));
    if (v) std::memcpy(v, c->h_stage + n3, n3 * sizeof(double));
    return BOUNCE_OK;
}

int bounce_run(bounce_ctx* c, int64_t n_steps, int32_t integ, void* stream) {
    if (!c) return BOUNCE_ERR_INVALID_ARG;
    if (!c->have_state) return fail(c, BOUNCE_ERR_STATE, "no state");
    int r = check_run_args(c, n_steps, integ);
    if (r) return r;
    if (n_steps == 0) return BOUNCE_OK;
    cudaSetDevice(c->cfg.device);
    cudaStream_t st = (cudaStream_t)stream;
    const int m = respa_period(c, integ);
    long long s0 = c->cur_step;
    rows_before_run(c, integ, st);
    // head: B/2 [J] A O A at the current step
    boundary(c, integ, 0, 0, s0, st);
    launch_advance_step(c->ds, 1, st);
    long long base = s0 + 1;
    int64_t rem = n_steps - 1;
    while (rem >= CHUNK) {
        const int phase = (int)(base % m);
        if ((r = ensure_graph(c, integ, phase))) return r;
        CU(cudaGraphLaunch(c->graph[integ][phase], st));
        rem -= CHUNK;
        base += CHUNK;
    }
    for (int64_t k = 0; k < rem; ++k) boundary(c, integ, 1, (int)k, base + k, st);
    if (rem) launch_advance_step(c->ds, rem, st);
    // tail: [J] B/2
    boundary(c, integ, 2, 0, s0 + n_steps, st);
    c->cur_step = s0 + n_steps;
    if (integ == BOUNCE_BAOAB && c->ds.cl.on) c->rows_check_due = true;
    rows_after_run(c, integ);
    CU(cudaGetLastError());
    return check_err(c, st);
}

int bounce_profile_steps(bounce_ctx* c, int64_t n_steps, int32_t integ, void* stream, double* kernel_ms,
                         int64_t* launches) {
    if (!c) return BOUNCE_ERR_INVALID_ARG;
    if (!c->have_state) return fail(c, BOUNCE_ERR_STATE, "no state");
    if (n_steps < 1 || !kernel_ms) return fail(c, BOUNCE_ERR_INVALID_ARG, "bad profile arguments");
    if (int r0 = check_run_args(c, n_steps, integ)) return r0;
    cudaSetDevice(c->cfg.device);
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<cudaEvent_t> ev(2 * (size_t)(n_steps + 1));
    for (auto& e : ev) CU(cudaEventCreate(&e));
    const long long s0 = c->cur_step;
    rows_before_run(c, integ, st);
    auto timed = [&](int k, int variant, int off, long long step) {
        bool pme;
        double hr, hout;
        plan(c, integ, variant, step, pme, hr, hout);
        rebuild_for(c, integ, off, st);
        if (pme) launch_pme(c->ds, c->pp, c->pme, off, st);
        cudaEventRecord(ev[2 * k], st);
        launch_step(run_view(c, integ), c->pp, integ, variant, off, hr, hout, st);
        cudaEventRecord(ev[2 * k + 1], st);
    };
    timed(0, 0, 0, s0);
    launch_advance_step(c->ds, 1, st);
    for (int64_t k = 0; k < n_steps - 1; ++k) timed((int)k + 1, 1, (int)k, s0 + 1 + k);
    if (n_steps > 1) launch_advance_step(c->ds, n_steps - 1, st);
    timed((int)n_steps, 2, 0, s0 + n_steps);
    c->cur_step = s0 + n_steps;
    if (integ == BOUNCE_BAOAB && c->ds.cl.on) c->rows_check_due = true;
    rows_after_run(c, integ);
    CU(cudaStreamSynchronize(st));
    double tot = 0.0;
    for (int64_t k = 0; k <= n_steps; ++k) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev[2 * k], ev[2 * k + 1]);
        tot += ms;
    }
    for (auto& e : ev) cudaEventDestroy(e);
    *kernel_ms = tot;
    if (launches) *launches = n_steps + 1;
    return check_err(c, st);
}

int bounce_profile_breakdown(bounce_ctx* c, int64_t n_steps, int32_t integ, void* stream, double* ms,
                             int64_t* groups) {
    if (!c) return BOUNCE_ERR_INVALID_ARG;
    if (!c->have_state) return fail(c, BOUNCE_ERR_STATE, "no state");
    if (n_steps < 1 || !ms) return fail(c, BOUNCE_ERR_INVALID_ARG, "bad profile arguments");
    if (int r0 = check_run_args(c, n_steps, integ)) return r0;
    cudaSetDevice(c->cfg.device);
    cudaStream_t st = (cudaStream_t)stream;
    constexpr int NK = 5;  // pair sums, step kernel, row rebuild, cluster rebuild, SPME
    std::vector<cudaEvent_t> ev;
    std::vector<int> kind;
    auto mark = [&](int k) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return false;
        cudaEventRecord(e, st);
        ev.push_back(e);
        kind.push_back(k);
        return true;
    };
    const long long s0 = c->cur_step;
    rows_before_run(c, integ, st);
    bool ok = true;
    auto one = [&](int variant, int off, long long step) {
        bool pme;
        double hr, hout;
        plan(c, integ, variant, step, pme, hr, hout);
        const DevSys v = run_view(c, integ);
        ok = ok && mark(-1);
        if (c->ds.cl.on) launch_cluster_rebuild(c->ds, c->pp, off, false, st);
        ok = ok && mark(3);
        if (!c->ds.cl.on || integ != BOUNCE_BAOAB) rebuild(c, off, false, st, run_rows_mode(c, integ));
        ok = ok && mark(2);
        if (pme) launch_pme(c->ds, c->pp, c->pme, off, st);
        ok = ok && mark(4);
        const int pre = launch_step_pairs(v, c->pp, integ, off, hout, st);
        ok = ok && mark(0);
        launch_step_kernel(v, c->pp, integ, variant, off, hr, hout, pre, st);
        ok = ok && mark(1);
    };
    one(0, 0, s0);
    launch_advance_step(c->ds, 1, st);
    for (int64_t k = 0; k < n_steps - 1; ++k) one(1, (int)k, s0 + 1 + k);
    if (n_steps > 1) launch_advance_step(c->ds, n_steps - 1, st);
    one(2, 0, s0 + n_steps);
    c->cur_step = s0 + n_steps;
    if (integ == BOUNCE_BAOAB && c->ds.cl.on) c->rows_check_due = true;
    rows_after_run(c, integ);
    CU(cudaStreamSynchronize(st));
    for (int k = 0; k < NK; ++k) {
        ms[k] = 0.0;
        if (groups) groups[k] = 0;
    }
    for (size_t e = 1; e < ev.size(); ++e) {
        if (kind[e] < 0) continue;
        float t = 0.f;
        cudaEventElapsedTime(&t, ev[e - 1], ev[e]);
        ms[kind[e]] += t;
        if (groups) groups[kind[e]] += 1;
    }
    for (auto& e : ev) cudaEventDestroy(e);
    if (!ok) return fail(c, BOUNCE_ERR_CUDA, "cudaEventCreate failed");
    return check_err(c, st);
}

int bounce_autotune(bounce_ctx* c, int32_t integ, void* stream, bounce_tuning* out) {
    if (!c || !out || integ < BOUNCE_BAOAB || integ > BOUNCE_BOUNCE_RESPA1)
        return fail(c, BOUNCE_ERR_INVALID_ARG, "bad autotune arguments");
    if (!c->have_state) return fail(c, BOUNCE_ERR_STATE, "no state");
    cudaSetDevice(c->cfg.device);
    cudaStream_t st = (cudaStream_t)stream;
    std::memset(out, 0, sizeof(*out));
    const int part = integ == BOUNCE_BAOAB ? 5 : 3;
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    constexpr int REPS = 5;
    auto time_pairs = [&](auto launch) -> double {
        launch();  // warm
        cudaEventRecord(e0, st);
        for (int k = 0; k < REPS; ++k) launch();
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms / REPS;
    };
    int r = BOUNCE_OK;
    if (c->ds.tl.on) {
        // tile kernel: j-block length x resident grid
        const int tjs[4] = {32, 64, 128, 256}, grids[3] = {152 * 2, 152 * 4, 152 * 8};
        double best = 1e30;
        int bj = c->tile_j, bg = c->tile_blocks;
        for (int tj : tjs)
            for (int gb : grids) {
                c->tile_j = tj;
                c->tile_blocks = gb;
                if ((r = setup_tiles(c))) break;
                const double ms = time_pairs([&] { launch_tile_pairs(c->ds, c->pp, 0, part, st); });
                ++out->candidates;
                if (ms < best) {
                    best = ms;
                    bj = tj;
                    bg = gb;
                }
            }
        c->tile_j = bj;
        c->tile_blocks = bg;
        if (!r) r = setup_tiles(c);
        CU(cudaMemsetAsync(c->ds.tl.acc, 0, 3 * (size_t)c->n * sizeof(unsigned long long), st));
        out->tile_j = bj;
        out->tile_blocks = bg;
        out->pair_ms = best;
    } else if (c->ds.cl.on) {
        // cluster columns: edge factor around (8 / density)^(1/3)
        std::vector<double> q(3 * (size_t)c->n);
        if ((r = bounce_get_state(c, q.data(), nullptr, BOUNCE_HOST, stream))) return r;
        const double fs[5] = {0.8, 0.9, 1.0, 1.12, 1.25};
        double best = 1e30, bf = c->cl_edge_factor;
        const int list = (part == 3 && c->ds.cl.nlists > 1) ? 1 : 0;
        for (double f : fs) {
            c->cl_edge_factor = f;
            c->cl_force = true;
            if ((r = setup_clusters(c, q.data()))) break;
            launch_cluster_rebuild(c->ds, c->pp, 0, true, st);
            const double ms = time_pairs([&] { launch_cluster_pairs(c->ds, c->pp, 0, part, list, st); });
            ++out->candidates;
            if (ms < best) {
                best = ms;
                bf = f;
            }
        }
        c->cl_edge_factor = bf;
        c->cl_force = true;
        if (!r) r = setup_clusters(c, q.data());
        if (!r) launch_cluster_rebuild(c->ds, c->pp, 0, true, st);
        const size_t ns = (size_t)c->ds.cl.ncol * c->ds.cl.maxcl * BOUNCE_CL;
        CU(cudaMemsetAsync(c->ds.cl.acc, 0, 3 * ns * sizeof(unsigned long long), st));
        out->column_edge = 1.0 / c->ds.cl.ihx;
        out->pair_ms = best;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    drop_graphs(c);
    CU(cudaStreamSynchronize(st));
    if (r) return r;
    return check_err(c, st);
}

int64_t bounce_run_launch_count(const bounce_ctx* c, int64_t n, int32_t integ) {
    if (!c || n <= 0) return 0;
    // gated row-rebuild kernels (cells count + scan, scatter, rows + flag clear;
    // one kernel for a batch of replicas) + the fused step kernel, and the
    // pair-sum kernel wherever the boundary has pair sums over the long rows
    const bool clu = c->ds.cl.on != 0;
    // gated rebuilds: the clusters (4, and the list prune), the rows (3, or 1
    // for a batch) unless BAOAB runs on clusters; then the step kernel
    const int64_t per_boundary = (clu ? 5 : 0) + ((clu && integ == BOUNCE_BAOAB) ? 0 : (c->ds.rep_of ? 1 : 3)) + 1;
    const bool ext = integ >= BOUNCE_BOUNCE_RESPA_EXT;
    const bool short_f0 = !clu && integ != BOUNCE_BAOAB && c->pp.rshort2 < INFINITY;
    const int64_t pme_launches = 10; // spread, load, 3 + 3 transforms, convolve, gather
    int64_t total = 2;               // step-counter updates after the head and the bodies
    for (int64_t k = 0; k <= n; ++k) {
        bool pme;
        double hr, hout;
        plan(c, integ, k == 0 ? 0 : (k == n ? 2 : 1), c->cur_step + k, pme, hr, hout);
        total += per_boundary + (pme ? pme_launches : 0) + (((ext && hout == 0.0) || short_f0) ? 0 : 1);
    }
    total += (n - 1) / CHUNK;        // one counter update per replayed graph chunk
    return total;
}

int bounce_get_energies(bounce_ctx* c, bounce_energies* out, void* stream) {
    if (!c || !out) return BOUNCE_ERR_INVALID_ARG;
    if (!c->have_state) return fail(c, BOUNCE_ERR_STATE, "no state");
    cudaSetDevice(c->cfg.device);
    cudaStream_t st = (cudaStream_t)stream;
    long long step;
    CU(cudaMemcpyAsync(&step, c->d_step, sizeof(long long), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    if (int r0 = prepare_readers(c, st)) return r0;
    launch_energies(c->ds, c->pp, (int)(step & 1), c->terms, st);
    double tot[5], pe[2] = {0.0, 0.0};
    if (c->has_pme) {
        launch_pme(c->ds, c->pp, c->pme, 0, st, true);
        launch_pme_energy(c->pme, c->n, c->terms + 6 * (size_t)c->n + 1024, st);
        CU(cudaMemcpyAsync(pe, c->terms + 6 * (size_t)c->n + 1024, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    CU(cudaMemcpyAsync(tot, c->terms + 5 * (size_t)c->n, 5 * sizeof(double), cudaMemcpyDeviceToHost, st));
    CU(cudaMemcpyAsync(c->h_cnt, c->ds.cnt, CNT_N * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    int r = check_err(c, st);
    if (r) return r;
    out->coulomb = KCOUL_D / (double)c->pp.kcoul * tot[0];
    out->lj = tot[1];
    out->bond = tot[2];
    out->angle = tot[3];
    out->kinetic = tot[4];
    out->recip = c->has_pme ? pe[0] + pe[1] + c->e_self : 0.0;
    out->potential = out->coulomb + out->lj + out->bond + out->angle + out->recip;
    out->temperature = 2.0 * tot[4] / (3.0 * c->n * KB_D);
    out->step = step - c->step0;
    out->proposals = (int64_t)c->h_cnt[CNT_PROPOSALS];
    out->accepts = (int64_t)c->h_cnt[CNT_ACCEPTS];
    out->near_ties = (int64_t)c->h_cnt[CNT_NEAR];
    out->rebuilds = (int64_t)c->h_cnt[CNT_REBUILDS];
    out->short_pairs = (int64_t)c->h_cnt[CNT_SHORT_PAIRS];
    out->full_pairs = (int64_t)c->h_cnt[CNT_FULL_PAIRS];
    return BOUNCE_OK;
}

int bounce_pair_histogram(bounce_ctx* c, int32_t ta, int32_t tb, double r_max, int32_t n_bins, int64_t* hist,
                          void* stream) {
    if (!c || !hist || n_bins < 1 || !(r_max > 0) || ta < 0 || tb < 0 || ta >= BOUNCE_MAXT || tb >= BOUNCE_MAXT)
        return fail(c, BOUNCE_ERR_INVALID_ARG, "bad histogram arguments");
    if (!c->have_state) return fail(c, BOUNCE_ERR_STATE, "no state");
    const bool cut = std::isfinite(c->cfg.r_cut) && c->cfg.r_cut > 0;
    if (cut && r_max > c->cfg.r_cut) return fail(c, BOUNCE_ERR_INVALID_ARG, "r_max exceeds the cutoff");
    cudaSetDevice(c->cfg.device);
    cudaStream_t st = (cudaStream_t)stream;
    if (n_bins > c->hist_alloc) {
        int r = dalloc(c, &c->hist, n_bins);
        if (r) return r;
        c->hist_alloc = n_bins;
    }
    long long step;
    CU(cudaMemcpyAsync(&step, c->d_step, sizeof(long long), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    if (int r0 = prepare_readers(c, st)) return r0;
    CU(cudaMemsetAsync(c->hist, 0, n_bins * sizeof(unsigned long long), st));
    launch_pair_hist(c->ds, c->pp, (int)(step & 1), ta, tb, r_max, n_bins, c->hist, st);
    CU(cudaMemcpyAsync(hist, c->hist, n_bins * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    return check_err(c, st);
}

int bounce_set_msd_reference(bounce_ctx* c, void* stream) {
    if (!c) return BOUNCE_ERR_INVALID_ARG;
    if (!c->have_state) return fail(c, BOUNCE_ERR_STATE, "no state");
    cudaSetDevice(c->cfg.device);
    cudaStream_t st = (cudaStream_t)stream;
    if (!c->msd_ref) {
        int r = dalloc(c, &c->msd_ref, 3 * (size_t)c->n);
        if (r) return r;
    }
    long long step;
    CU(cudaMemcpyAsync(&step, c->d_step, sizeof(long long), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    const int cur = (int)(step & 1);
    const size_t b = c->n * sizeof(double);
    CU(cudaMemcpyAsync(c->msd_ref, c->ds.qx[cur], b, cudaMemcpyDeviceToDevice, st));
    CU(cudaMemcpyAsync(c->msd_ref + c->n, c->ds.qy[cur], b, cudaMemcpyDeviceToDevice, st));
    CU(cudaMemcpyAsync(c->msd_ref + 2 * (size_t)c->n, c->ds.qz[cur], b, cudaMemcpyDeviceToDevice, st));
    CU(cudaStreamSynchronize(st));
    c->have_msd_ref = true;
    return BOUNCE_OK;
}

int bounce_msd(bounce_ctx* c, int32_t type, double* out, void* stream) {
    if (!c || !out || type < 0 || type >= BOUNCE_MAXT) return fail(c, BOUNCE_ERR_INVALID_ARG, "bad msd arguments");
    if (!c->have_msd_ref) return fail(c, BOUNCE_ERR_STATE, "no msd reference");
    cudaSetDevice(c->cfg.device);
    cudaStream_t st = (cudaStream_t)stream;
    long long step;
    CU(cudaMemcpyAsync(&step, c->d_step, sizeof(long long), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    launch_msd(c->ds, c->msd_ref, c->msd_ref + c->n, c->msd_ref + 2 * (size_t)c->n, (int)(step & 1), type, c->terms,
               st);
    double tot[2];
    CU(cudaMemcpyAsync(tot, c->terms + 2 * (size_t)c->n, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    *out = tot[1] > 0 ? tot[0] / tot[1] : 0.0;
    return BOUNCE_OK;
}

int bounce_reset_counters(bounce_ctx* c, void* stream) {
    if (!c) return BOUNCE_ERR_INVALID_ARG;
    if (!c->have_topo) return fail(c, BOUNCE_ERR_STATE, "no topology");
    cudaSetDevice(c->cfg.device);
    CU(cudaMemsetAsync(c->ds.cnt, 0, CNT_N * sizeof(unsigned long long), (cudaStream_t)stream));
    return BOUNCE_OK;
}

int bounce_get_bounds(bounce_ctx* c, double* L, double* Lstar) {
    if (!c) return BOUNCE_ERR_INVALID_ARG;
    if (!c->have_lj) return fail(c, BOUNCE_ERR_STATE, "no LJ table");
    const int T = c->n_types;
    if (L)
        for (int k = 0; k < T * T; ++k) L[k] = c->L[k];
    if (Lstar)
        for (int k = 0; k < T; ++k) Lstar[k] = c->Lstar[k];
    return BOUNCE_OK;
}

int bounce_compute_gradient(bounce_ctx* c, int32_t part, double* grad, int32_t where, void* stream) {
    if (!c || !grad || part < 0 || part > 3 || (where != BOUNCE_HOST && where != BOUNCE_DEVICE))
        return fail(c, BOUNCE_ERR_INVALID_ARG, "bad gradient arguments");
    if (!c->have_state) return fail(c, BOUNCE_ERR_STATE, "no state");
    cudaSetDevice(c->cfg.device);
    cudaStream_t st = (cudaStream_t)stream;
    long long step;
    CU(cudaMemcpyAsync(&step, c->d_step, sizeof(long long), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    if (int r0 = prepare_readers(c, st)) return r0;
    const cudaMemcpyKind kind = where == BOUNCE_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (part == BOUNCE_GRAD_RECIP) {
        if (!c->has_pme) return fail(c, BOUNCE_ERR_STATE, "no SPME grid configured");
        launch_pme(c->ds, c->pp, c->pme, 0, st);
        for (int d = 0; d < 3; ++d)
            CU(cudaMemcpy2DAsync(grad + d, 3 * sizeof(double), c->pme.grad + (size_t)d * c->n, sizeof(double),
                                 sizeof(double), c->n, kind, st));
    } else if (c->ds.tl.on && (part == BOUNCE_GRAD_FULL || (part == BOUNCE_GRAD_SHORT && !(c->pp.rshort2 < INFINITY)))) {
        // bonded terms, then the all-pairs tile sums added (the run's kernels)
        double* out = c->terms;
        launch_gradient(c->ds, c->pp, 4, (int)(step & 1), out, st);
        launch_tile_pairs(c->ds, c->pp, 0, part == BOUNCE_GRAD_FULL ? 5 : 3, st);
        launch_tile_collect(c->ds, out, st);
        CU(cudaMemcpyAsync(grad, out, 3 * (size_t)c->n * sizeof(double), kind, st));
    } else if (c->ds.cl.on && part != BOUNCE_GRAD_LONG) {
        // bonded terms, then the cluster pair sums added (the run's kernels)
        double* out = c->terms;
        launch_cluster_rebuild(c->ds, c->pp, 0, false, st);
        launch_gradient(c->ds, c->pp, 4, (int)(step & 1), out, st);
        const bool full = part == BOUNCE_GRAD_FULL;
        launch_cluster_pairs(c->ds, c->pp, 0, full ? 5 : 3, (!full && c->ds.cl.nlists > 1) ? 1 : 0, st);
        launch_cluster_collect(c->ds, out, st);
        CU(cudaMemcpyAsync(grad, out, 3 * (size_t)c->n * sizeof(double), kind, st));
    } else {
        double* out = c->terms;  // scratch of 6 n doubles >= 3 n
        launch_gradient(c->ds, c->pp, part, (int)(step & 1), out, st);
        CU(cudaMemcpyAsync(grad, out, 3 * (size_t)c->n * sizeof(double), kind, st));
    }
    CU(cudaStreamSynchronize(st));
    return check_err(c, st);
}

int bounce_jump_half(bounce_ctx* c, int64_t step, int32_t stream_id, int32_t* M, int32_t* nacc, int32_t where,
                     void* stream) {
    if (!c || step < 0 || stream_id < 0 || stream_id > 255 || (where != BOUNCE_HOST && where != BOUNCE_DEVICE))
        return fail(c, BOUNCE_ERR_INVALID_ARG, "bad jump arguments");
    if (!c->have_state) return fail(c, BOUNCE_ERR_STATE, "no state");
    cudaSetDevice(c->cfg.device);
    cudaStream_t st = (cudaStream_t)stream;
    long long cur_step;
    CU(cudaMemcpyAsync(&cur_step, c->d_step, sizeof(long long), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    if (c->jfilter) {
        // the stand-alone half-step draws over the full rows
        if (int r0 = prepare_readers(c, st)) return r0;
    } else {
        rebuild(c, 0, false, st);
    }
    int* dM = nullptr;
    int* dA = nullptr;
    if (M || nacc) {
        int* tmp = (int*)c->terms;  // 12 n ints of scratch
        dM = tmp;
        dA = tmp + c->n;
    }
    launch_jump_half(c->ds, c->pp, (int)(cur_step & 1), step, stream_id, dM, dA, st);
    const cudaMemcpyKind kind = where == BOUNCE_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (M) CU(cudaMemcpyAsync(M, dM, c->n * sizeof(int), kind, st));
    if (nacc) CU(cudaMemcpyAsync(nacc, dA, c->n * sizeof(int), kind, st));
    CU(cudaStreamSynchronize(st));
    return check_err(c, st);
}

int bounce_get_rows(bounce_ctx* c, int32_t* counts, int32_t* rows, int32_t capacity) {
    if (!c || !counts || !rows || capacity < 1) return fail(c, BOUNCE_ERR_INVALID_ARG, "bad row arguments");
    if (!c->have_state) return fail(c, BOUNCE_ERR_STATE, "no state");
    cudaSetDevice(c->cfg.device);
    if (int r0 = prepare_readers(c, nullptr)) return r0;
    CU(cudaDeviceSynchronize());
    int r = check_err(c, nullptr);
    if (r) return r;
    const int n = c->n, cap = c->ds.cap;
    std::vector<int> cnt(n), all((size_t)n * cap);
    CU(cudaMemcpy(cnt.data(), c->ds.nlong, n * sizeof(int), cudaMemcpyDeviceToHost));
    CU(cudaMemcpy(all.data(), c->ds.rows, all.size() * sizeof(int), cudaMemcpyDeviceToHost));
    for (int i = 0; i < n; ++i) {
        counts[i] = cnt[i];
        for (int k = 0; k < std::min(cnt[i], capacity); ++k) rows[(size_t)i * capacity + k] = all[(size_t)i * cap + k];
    }
    return BOUNCE_OK;
}

int bounce_set_replicas(bounce_ctx* c, int32_t n_rep, const int32_t* off, const uint64_t* seeds) {
    if (!c || n_rep < 1 || !off || !seeds) return fail(c, BOUNCE_ERR_INVALID_ARG, "bad replica arguments");
    if (!c->have_topo) return fail(c, BOUNCE_ERR_STATE, "set the topology first");
    if (c->cfg.periodic || (std::isfinite(c->cfg.r_cut) && c->cfg.r_cut > 0))
        return fail(c, BOUNCE_ERR_UNSUPPORTED, "replica batches are open droplets without a cutoff");
    if (off[0] != 0 || off[n_rep] != c->n) return fail(c, BOUNCE_ERR_INVALID_ARG, "offsets must cover all atoms");
    std::vector<int> rep(c->n), loc(c->n);
    int maxn = 0;
    for (int r = 0; r < n_rep; ++r) {
        if (off[r + 1] <= off[r]) return fail(c, BOUNCE_ERR_INVALID_ARG, "empty or unordered replica");
        maxn = std::max(maxn, off[r + 1] - off[r]);
        for (int i = off[r]; i < off[r + 1]; ++i) {
            rep[i] = r;
            loc[i] = i - off[r];
        }
    }
    // a molecule must not span two replicas
    std::vector<int> mol_rep;
    for (int i = 0; i < c->n; ++i) {
        const int m = c->mol[i];
        if (m >= (int)mol_rep.size()) mol_rep.resize(m + 1, -1);
        if (mol_rep[m] >= 0 && mol_rep[m] != rep[i]) return fail(c, BOUNCE_ERR_INVALID_ARG, "molecule spans replicas");
        mol_rep[m] = rep[i];
    }
    if (maxn - 1 > c->ds.cap) return fail(c, BOUNCE_ERR_INVALID_ARG, "max_neighbors below the largest replica size - 1");
    cudaSetDevice(c->cfg.device);
    std::vector<uint2> keys(n_rep);
    for (int r = 0; r < n_rep; ++r) keys[r] = make_uint2((uint32_t)(seeds[r] & 0xFFFFFFFFull), (uint32_t)(seeds[r] >> 32));
    int *drep, *dloc, *doff;
    uint2* dkey;
    int rr;
    if ((rr = dalloc(c, &drep, c->n)) || (rr = dalloc(c, &dloc, c->n)) || (rr = dalloc(c, &doff, n_rep + 1)) ||
        (rr = dalloc(c, &dkey, n_rep)))
        return rr;
    CU(cudaMemcpy(drep, rep.data(), c->n * sizeof(int), cudaMemcpyHostToDevice));
    CU(cudaMemcpy(dloc, loc.data(), c->n * sizeof(int), cudaMemcpyHostToDevice));
    CU(cudaMemcpy(doff, off, (n_rep + 1) * sizeof(int), cudaMemcpyHostToDevice));
    CU(cudaMemcpy(dkey, keys.data(), n_rep * sizeof(uint2), cudaMemcpyHostToDevice));
    c->ds.rep_of = drep;
    c->ds.local_idx = dloc;
    c->ds.rep_off = doff;
    c->ds.rep_key = dkey;
    c->rep_bounds.assign(off, off + n_rep + 1);
    if ((rr = setup_tiles(c))) return rr;
    drop_graphs(c);
    c->rows_valid = false;
    set_rows_kind(c, 0);
    ++c->pos_version;
    return BOUNCE_OK;
}

// Per-type parameters as FP32 tables, sigma and eps symmetrised from the
// upper triangle (entry (a, b) with a <= b is the parameter of the pair).
static int diff_tables(bounce_ctx* c, int32_t T, const double* qt, const double* sig, const double* eps, float* fq,
                       float* fs, float* fe) {
    if (T < c->n_types || T > BOUNCE_MAXT || !qt || !sig || !eps)
        return fail(c, BOUNCE_ERR_INVALID_ARG, "bad parameter tables");
    for (int a = 0; a < BOUNCE_MAXT; ++a) fq[a] = a < T ? (float)qt[a] : 0.f;
    for (int a = 0; a < BOUNCE_MAXT * BOUNCE_MAXT; ++a) fs[a] = fe[a] = 0.f;
    for (int a = 0; a < T; ++a)
        for (int b = 0; b < T; ++b) {
            const int lo = std::min(a, b), hi = std::max(a, b);
            fs[a * BOUNCE_MAXT + b] = (float)sig[lo * T + hi];
            fe[a * BOUNCE_MAXT + b] = (float)eps[lo * T + hi];
        }
    return BOUNCE_OK;
}

int bounce_pair_forward(bounce_ctx* c, const double* q, int32_t T, const double* qt, const double* sig,
                        const double* eps, double* forces, double* energy, void* stream) {
    if (!c || !forces) return fail(c, BOUNCE_ERR_INVALID_ARG, "bad forward arguments");
    if (!c->have_state) return fail(c, BOUNCE_ERR_STATE, "no state");
    float fq[BOUNCE_MAXT], fs[BOUNCE_MAXT * BOUNCE_MAXT], fe[BOUNCE_MAXT * BOUNCE_MAXT];
    int r = diff_tables(c, T, qt, sig, eps, fq, fs, fe);
    if (r) return r;
    cudaSetDevice(c->cfg.device);
    cudaStream_t st = (cudaStream_t)stream;
    const int cur = (int)(c->cur_step & 1);
    const int n = c->n;
    if (q) {
        CU(cudaMemcpy2DAsync(c->ds.qx[cur], sizeof(double), q + 0, 3 * sizeof(double), sizeof(double), n,
                             cudaMemcpyDeviceToDevice, st));
        CU(cudaMemcpy2DAsync(c->ds.qy[cur], sizeof(double), q + 1, 3 * sizeof(double), sizeof(double), n,
                             cudaMemcpyDeviceToDevice, st));
        CU(cudaMemcpy2DAsync(c->ds.qz[cur], sizeof(double), q + 2, 3 * sizeof(double), sizeof(double), n,
                             cudaMemcpyDeviceToDevice, st));
        launch_pack_positions(c->ds, c->pp, cur, st);
        if ((r = flag_clusters(c, st))) return r;
        if ((r = prepare_readers(c, st, true))) return r;
    } else {
        if ((r = prepare_readers(c, st))) return r;
    }
    double* eatom = c->terms;
    double* esum = c->terms + 6 * (size_t)n + 1024;
    launch_pair_forward(c->ds, c->pp, fq, fs, fe, T, cur, forces, eatom, esum, st);
    double e = 0.0;
    CU(cudaMemcpyAsync(&e, esum, sizeof(double), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    if (energy) *energy = e;
    return check_err(c, st);
}

int bounce_pair_backward(bounce_ctx* c, int32_t T, const double* qt, const double* sig, const double* eps,
                         const double* grad_forces, double grad_energy, double* grad_pos, double* grad_qt,
                         double* grad_sig, double* grad_eps, void* stream) {
    if (!c || !grad_forces || !grad_pos) return fail(c, BOUNCE_ERR_INVALID_ARG, "bad backward arguments");
    if (!c->have_state) return fail(c, BOUNCE_ERR_STATE, "no state");
    float fq[BOUNCE_MAXT], fs[BOUNCE_MAXT * BOUNCE_MAXT], fe[BOUNCE_MAXT * BOUNCE_MAXT];
    int r = diff_tables(c, T, qt, sig, eps, fq, fs, fe);
    if (r) return r;
    cudaSetDevice(c->cfg.device);
    cudaStream_t st = (cudaStream_t)stream;
    const int np = diff_param_count();
    if (!c->diff_part && (r = dalloc(c, &c->diff_part, (size_t)np * c->n + np))) return r;
    const int cur = (int)(c->cur_step & 1);
    double* psum = c->diff_part + (size_t)np * c->n;
    launch_pair_backward(c->ds, c->pp, fq, fs, fe, T, cur, grad_forces, grad_energy, grad_pos, c->diff_part, psum, st);
    std::vector<double> ps(np);
    CU(cudaMemcpyAsync(ps.data(), psum, np * sizeof(double), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    const int M = BOUNCE_MAXT;
    for (int a = 0; a < T; ++a) {
        if (grad_qt) grad_qt[a] = ps[a];
        for (int b = 0; b < T; ++b) {
            const int lo = std::min(a, b), hi = std::max(a, b);
            if (grad_sig) grad_sig[a * T + b] = ps[M + lo * M + hi];
            if (grad_eps) grad_eps[a * T + b] = ps[M + M * M + lo * M + hi];
        }
    }
    return check_err(c, st);
}

const char* bounce_last_error(const bounce_ctx* c) {
    if (!c) return "null context";
    return c->err.c_str();
}

void bounce_destroy(bounce_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->cfg.device);
    free_all(c);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->h_err) cudaFreeHost(c->h_err);
    if (c->h_cnt) cudaFreeHost(c->h_cnt);
    delete c;
}

}  // extern "C"
