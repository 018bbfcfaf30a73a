// libtdgl host runtime: contexts, simulations, batches and the C ABI declared in include/tdgl.h.
//
// One explicit TDGL step (Eq. 1, forward Euler, L = 1) of a sim whose electrostatic term is on is
//   [k_yfwd, k_zconv, k_yinv]  x-spectrum of P  ->  x-spectrum of E_el  (Eqs. 5-6)
//   k_rows<STEP>               E_el rows, Landau (Eq. 3), gradient (Eq. 4), E_ext (Eq. 7),
//                              update, and the x-spectrum of the new P for the next step.
// A batch issues each of these kernels once over the work items of all of its sims.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <tuple>
#include <utility>
#include <vector>

#include "../../include/tdgl.h"
#include "kernels.cuh"
#include "kernels_fast.cuh"
#include "kernels_rows.cuh"
#include "tensor.cuh"
#include "runtime.cuh"

using namespace tdgl;
using namespace tdgl_rt;

namespace {

const double kEps0 = 8.8541878128e-12;   // F/m
const int kMaxSmem = 200 * 1024;
constexpr int kZVariants = TDGL_ZPASS_VARIANTS;

enum { XS_NONE = 0, XS_PHAT = 1, XS_EHAT = 2 };


}  // namespace

struct tdgl_sim {
    tdgl_ctx *ctx = nullptr;
    int nx = 0, ny = 0, nz = 0;
    double d[3] = {0, 0, 0};
    long ncell = 0;
    int Mx = 0, My = 0, Mz = 0, hx = 0, Kx = 0, kxp = 0, kyh = 0, kzh = 0;
    tdgl_material mats[TDGL_MAX_MATERIALS];
    bool defined[TDGL_MAX_MATERIALS] = {false};
    std::vector<uint8_t> map;
    double T = 300.0, eps_b = 1.0, E[3] = {0, 0, 0};
    double Eac[3] = {0, 0, 0}, ac_freq = 0.0, ac_phase = 0.0;   // E_ext(t) = E + Eac sin(2 pi f t + phase)
    double time = 0.0;                                          // simulated time, s
    int integrator = TDGL_EULER;
    float *dhbuf = nullptr;                                     // Heun: first field evaluation
    float *dstage = nullptr;                                    // RK45 / AB3M2: 6 x 3N field evaluations
    CUtensorMap ymap;                                           // TMA view of dY for the z pass
    bool has_ymap = false;
    CUtensorMap nmap;                                           // TMA view of dNhat (staged z pass)
    bool has_nmap = false;
    unsigned *derrmax = nullptr;                                // RK45: max local error (float bits)
    double ad_tol = 0.0, ad_min = 0.0, ad_max = 0.0, dt_next = 0.0;   // RK45 step-size control
    int ab_hist = 0, ab_ring = 0;                               // AB3M2: valid history, newest slot
    unsigned terms = TDGL_TERM_ALL;
    double P0 = 1.0, alpha_ref = 1.0;
    bool scales_fixed = false;
    double ell = 1.0;   // length unit: smallest cell edge
    // device buffers
    float *dP[2] = {nullptr, nullptr};
    uint8_t *dmat = nullptr;
    float2 *dX = nullptr, *dY = nullptr;
    float2 *dNhat = nullptr;
    float2 *dtw = nullptr;
    float *dcoef = nullptr;
    unsigned *dmaxdp = nullptr;
    int *dflag = nullptr;
    double *denergy = nullptr;
    float *dout = nullptr;
    SimDev *ddesc = nullptr;
    SimDev desc;
    Plan px, py, pz;
    int twr = 0;
    // work items
    std::vector<int4> it_rows, it_y, it_z;
    std::vector<int4> it_rows_full;   // row items of full tiles (batches)
    int rows_cnt_max = 1, ky_cnt_max = 1, kz_cnt_max = 1;
    int xN = 0, yN = 0, zN = 0;   // specialized x / y / z transform length (0 = generic kernels)
    // rows per block of the tiled row kernel when the sim runs alone: 0 = the size heuristic,
    // else the autotuner's choice; the candidates it timed and their microseconds per launch
    int row_tile = 0;
    bool rows_tuned = false;
    int row_cand[TDGL_ROW_CANDIDATES] = {0};
    double row_us[TDGL_ROW_CANDIDATES] = {0.0};
    int4 *d_rows = nullptr, *d_y = nullptr, *d_z = nullptr;
    int cur = 0;
    int xstate = XS_NONE;
    bool spectra_alloc = false, tensor_ready = false;
    bool has_cross = false;
    bool dirty = true;      // map, materials, T or scales changed since the last prepare()
    struct GraphRec { int n; bool elec; int p0; int integ; cudaGraphExec_t exec; long kernels; };
    std::vector<GraphRec> graphs;   // captured steady step sequences
    std::vector<GraphRec> relax_graphs;   // device-side relaxation loops (n = steps per chunk)
    RelaxState *drelax = nullptr;         // their loop state
    double last_maxdp = 0.0;
    tdgl_batch *batch = nullptr;
    // asynchronous host I/O: two staging buffers per direction, used in turn, and the events that
    // order each (input landed, input consumed, output staged, output read out); status of steps
    // that tdgl_step_async enqueued and nobody has read yet
    float *din_a[2] = {nullptr, nullptr}, *dout_a[2] = {nullptr, nullptr};
    cudaEvent_t ev_in_ready[2] = {}, ev_in_free[2] = {}, ev_out_ready[2] = {}, ev_out_free[2] = {};
    int in_next = 0, out_next = 0;
    bool status_pending = false;
};

// loop state of a batch's device relaxation: steps done in this launch's loop, the cap, the
// tolerance, steps per body, batch size, and the cells retired so far against the cells after which
// the loop hands back to the host (which then drops the retired sims from the work lists)
struct BatchRelaxState {
    long done, max_steps;
    double tol;
    int k, n;
    long cells_retired, cells_stop;
};

struct tdgl_batch {
    tdgl_ctx *ctx = nullptr;
    std::vector<tdgl_sim *> sims;
    SimDev *ddescs = nullptr;
    int4 *d_items = nullptr;
    size_t items_cap = 0;
    // work lists and captured step sequences for the current active set
    std::vector<int> w_active;
    struct Cached;
    Cached *cache = nullptr;
    // device relaxation loop state: loop counters, membership of the current active set, steps
    // taken and status (0 running, 1 converged, 2 diverged, 3 a bounded wait timed out) per sim
    struct BatchRelaxState *drelax = nullptr;
    int *dmember = nullptr, *dstatus = nullptr;
    long *dsteps = nullptr;
};

// frees a batch's cached work lists and graphs (defined once the cache type is complete)
static void drop_cache(tdgl_batch *b);

// ---------------------------------------------------------------------------------------------
namespace {




int smooth_at_least(int m, bool even) {
    // smallest 2^a 3^b >= m (even when asked)
    int best = 1 << 30;
    for (long p2 = 1; p2 < (1L << 30); p2 *= 2)
        for (long v = p2; v < (1L << 30); v *= 3) {
            if (v >= m && (!even || v % 2 == 0) && v < best) best = (int)v;
            if (v >= m) break;
        }
    return best;
}

bool is_smooth(int m) {   // m = 2^a 3^b
    if (m < 1) return false;
    while (m % 2 == 0) m /= 2;
    while (m % 3 == 0) m /= 3;
    return m == 1;
}

// smallest length >= m that the specialized (register) transforms cover, 0 if none
int fast_at_least(int m) {
    static const int L[] = {16, 32, 48, 64, 96, 128, 192, 256, 512};
    for (int v : L)
        if (v >= m) return v;
    return 0;
}

// Default padded length of the y or z axis of n cells: the smallest 2^a 3^b >= 2n - 1, except
//  - along z, a length with a factor 3 gives way to the next power of two when that is one of the
//    z pass's tuned lengths (128, 256, 512) and at most 4/3 of it (96 -> 128, 192 -> 256, 384 ->
//    512): the tuned 256-point z pass takes 15 ps per point against 29 ps for the 192-point shape;
//  - a length the specialized transforms do not cover gives way to the smallest one they cover
//    when that is at most 4/3 of it (81 -> 96, 162 -> 192): the generic shared-memory kernels take
//    2-3 times as long per point (80^3 cube: 407 -> 221 us per step).
// Any length >= 2n - 1 gives the same linear convolution.
int default_yz_length(int n, bool z) {
    const int m = smooth_at_least(2 * n - 1, false);
    if (z && m % 3 == 0) {
        int p2 = 1;
        while (p2 < m) p2 *= 2;
        if ((p2 == 128 || p2 == 256 || p2 == 512) && 3 * p2 <= 4 * m) return p2;
    }
    const int f = fast_at_least(2 * n - 1);
    return (f && f != m && 3 * f <= 4 * m && fast_at_least(m) != m) ? f : m;
}
int default_z_length(int nz) { return default_yz_length(nz, true); }
int default_y_length(int ny) { return default_yz_length(ny, false); }

// Default padded length of the x axis of nx cells: the smallest even 2^a 3^b >= 2 nx - 1, except
// that when its half is not a specialized length and nx is a multiple of 4 it gives way to twice the
// smallest specialized half-length >= nx within 4/3 (80 cells: 162 -> 192), so the rows run in the
// tiled step kernel (which takes rows of nx <= Mx / 2 cells, nx a multiple of 4) instead of the
// generic one.
int default_x_length(int nx) {
    const int m = smooth_at_least(2 * nx - 1, true);
    if (nx % 4 != 0 || fast_at_least(m / 2) == m / 2) return m;
    const int h = fast_at_least(nx);
    return (h && 3 * (2 * h) <= 4 * m) ? 2 * h : m;
}

Plan make_plan(int n, std::vector<float2> &tw) {
    Plan p;
    memset(&p, 0, sizeof p);
    p.n = n;
    int r = n;
    const int rads[5] = {16, 8, 4, 3, 2};
    for (int i = 0; i < 5; ++i)
        while (r % rads[i] == 0 && r > 1) {
            p.rad[p.nrad++] = rads[i];
            r /= rads[i];
        }
    p.tw = (int)tw.size();
    for (int t = 0; t < n; ++t) {
        const double a = -2.0 * M_PI * (double)t / (double)n;
        tw.push_back(make_float2((float)cos(a), (float)sin(a)));
    }
    return p;
}

double alpha1_of(const tdgl_material &m, double T) {
    if (m.a1_form == 1) {
        auto coth = [](double v) { return cosh(v) / sinh(v); };
        return m.coth_A * (coth(m.coth_Ts / T) - coth(m.coth_Ts / m.coth_T1));
    }
    if (m.a1_form == 2) return m.a0;
    return m.a0 * (T - m.T0);
}

// tetragonal spontaneous polarization of a material at T (Eq. 12 along <100>), 0 if none
double tetragonal_ps(const tdgl_material &m, double T) {
    const double a1 = alpha1_of(m, T);
    const double a11 = m.a11_0 + m.a11_T * (T - m.a11_Tref);
    const double a111 = m.a111_0 + m.a111_T * (T - m.a111_Tref);
    // 2 a1 + 4 a11 u + 6 a111 u^2 = 0, u = P^2, minimum: 4 a11 + 12 a111 u > 0
    double best = 0.0, fbest = 0.0;
    double roots[2];
    int nr = 0;
    if (a111 != 0.0) {
        const double disc = 16.0 * a11 * a11 - 48.0 * a111 * a1;
        if (disc >= 0) {
            roots[nr++] = (-4.0 * a11 + sqrt(disc)) / (12.0 * a111);
            roots[nr++] = (-4.0 * a11 - sqrt(disc)) / (12.0 * a111);
        }
    } else if (a11 != 0.0) {
        roots[nr++] = -a1 / (2.0 * a11);
    }
    for (int i = 0; i < nr; ++i) {
        const double u = roots[i];
        if (!(u > 0) || 4.0 * a11 + 12.0 * a111 * u <= 0) continue;
        const double f = a1 * u + a11 * u * u + a111 * u * u * u;
        if (f < fbest) { fbest = f; best = sqrt(u); }
    }
    return best;
}




// Record the launches issued by record() into a CUDA graph and instantiate it.  The launches are
// not counted at capture time; *kernels receives how many each replay issues.
template <class F>
int capture_graph(tdgl_ctx *ctx, F record, cudaGraphExec_t *out, long *kernels) {
    const long l0 = ctx->launches;
    CK(ctx, cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    const int rc = record();
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
    *kernels = ctx->launches - l0;
    ctx->launches = l0;
    if (rc != TDGL_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    CK(ctx, e);
    const cudaError_t e2 = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    CK(ctx, e2);
    return TDGL_OK;
}

int grid_for(long n) { return (int)std::min<long>(std::max<long>((n + 255) / 256, 1), 148L * 16); }

// -- geometry and plans ------------------------------------------------------------------------
// lengths with a register-FFT specialization (fft_reg.cuh); the host reads each kernel's
// geometry from the same constexpr functions the kernels are compiled with
#define TDGL_FAST_LENGTHS(X) X(16) X(32) X(64) X(128) X(256) X(512) X(48) X(96) X(192)
bool fast_len(int n) {
    switch (n) {
#define TDGL_C(LEN) case LEN:
        TDGL_FAST_LENGTHS(TDGL_C)
#undef TDGL_C
        return true;
    }
    return false;
}
int fast_rowtile(int n) {   // rows per block of the tiled row kernel
    switch (n) {
#define TDGL_C(LEN) case LEN: return xrows_tile<LEN>();
        TDGL_FAST_LENGTHS(TDGL_C)
#undef TDGL_C
    }
    return 0;
}
int fast_ylines(int n) {    // lines per block of the y pass
    switch (n) {
#define TDGL_C(LEN) case LEN: return lines_per_block<LEN>();
        TDGL_FAST_LENGTHS(TDGL_C)
#undef TDGL_C
    }
    return 0;
}
int fast_zlines(int n) {    // lines per block of the z pass
    switch (n) {
#define TDGL_C(LEN) case LEN: return zlines_per_block<LEN, 0>();
        TDGL_FAST_LENGTHS(TDGL_C)
#undef TDGL_C
    }
    return 0;
}

void build_items(tdgl_sim *s) {
    s->it_rows.clear();
    s->it_rows_full.clear();
    s->it_y.clear();
    s->it_z.clear();
    // the tiled row kernel takes rows of nx <= hx cells, nx a multiple of 4 (a shorter row is zero
    // padded inside its x transforms)
    s->xN = (fast_len(s->hx) && s->nx <= s->hx && s->nx % 4 == 0) ? s->hx : 0;
    const int RB = s->xN ? fast_rowtile(s->hx)
                         : std::max(1, std::min(s->ny, std::max(1, 512 / s->nx)));
    s->rows_cnt_max = RB;
    // A sim run alone whose full tiles would give fewer blocks than SMs takes fewer rows per block,
    // about one block per SM (such a small grid is bound by each block's latency, not by the
    // tile's halo overhead); in a batch the members' full tiles already fill the GPU.
    const long rows = (long)s->ny * s->nz;
    const int RB1 = s->row_tile > 0 ? std::min(s->row_tile, RB)
                    : (s->xN ? (int)std::min<long>(RB, std::max<long>(1, (rows + s->ctx->nsm - 1) / s->ctx->nsm)) : RB);
    for (int z = 0; z < s->nz; ++z) {
        for (int y0 = 0; y0 < s->ny; y0 += RB1) s->it_rows.push_back(make_int4(0, z, y0, std::min(RB1, s->ny - y0)));
        for (int y0 = 0; y0 < s->ny; y0 += RB) s->it_rows_full.push_back(make_int4(0, z, y0, std::min(RB, s->ny - y0)));
    }
    s->yN = fast_len(s->My) ? s->My : 0;
    s->zN = fast_len(s->Mz) ? s->Mz : 0;
    // Kx = Mx/2 + 1 columns: when the first Mx/2 fill whole line groups, the last (Nyquist) column
    // would be a group of one line; the fast kernels instead take it in "across" items whose lanes
    // run over rows (cz for y, ky for z) of that column (flag kAcross in .w).
    const int ky = s->yN ? fast_ylines(s->My) : std::max(1, std::min(16, 73728 / (16 * (s->My + 1))));
    s->ky_cnt_max = ky;
    const bool y_across = s->yN && s->Kx > 1 && (s->Kx - 1) % ky == 0;
    const int ky_cols = y_across ? s->Kx - 1 : s->Kx;
    // the across items (uncoalesced, so slower per block) go first: they start in the first wave
    // instead of trailing behind the last one
    if (y_across)
        for (int r0 = 0; r0 < 3 * s->nz; r0 += ky)
            s->it_y.push_back(make_int4(0, r0, s->Kx - 1, std::min(ky, 3 * s->nz - r0) | kAcross));
    for (int c = 0; c < 3; ++c)
        for (int z = 0; z < s->nz; ++z)
            for (int k0 = 0; k0 < ky_cols; k0 += ky)
                s->it_y.push_back(make_int4(0, c * s->nz + z, k0, std::min(ky, ky_cols - k0)));
    const int kz = s->zN ? fast_zlines(s->Mz) : std::max(1, std::min(16, 102400 / (48 * (s->Mz + 1))));
    s->kz_cnt_max = kz;
    const bool z_across = s->zN && s->Kx > 1 && (s->Kx - 1) % kz == 0;
    const int kz_cols = z_across ? s->Kx - 1 : s->Kx;
    // rows ky and My - ky read the same tensor row: issue them back to back so the second read hits L2
    std::vector<int> order;
    for (int k = 0; k <= s->My / 2; ++k) {
        order.push_back(k);
        if (k != 0 && s->My - k != k) order.push_back(s->My - k);
    }
    if (z_across)
        for (int r0 = 0; r0 < s->My; r0 += kz)
            s->it_z.push_back(make_int4(0, r0, s->Kx - 1, std::min(kz, s->My - r0) | kAcross));
    for (int k : order)
        for (int k0 = 0; k0 < kz_cols; k0 += kz) s->it_z.push_back(make_int4(0, k, k0, std::min(kz, kz_cols - k0)));
}

size_t xrows_smem_for(int hx) {
    switch (hx) {
#define TDGL_XS(LEN) case LEN: return xrows_smem<LEN>();
        TDGL_XS(16) TDGL_XS(32) TDGL_XS(64) TDGL_XS(128) TDGL_XS(256) TDGL_XS(512) TDGL_XS(48) TDGL_XS(96) TDGL_XS(192)
#undef TDGL_XS
    }
    return 0;
}
size_t smem_rows(const tdgl_sim *s, int cnt) {
    return s->xN ? xrows_smem_for(s->xN) : 2ull * 3 * cnt * (s->hx + 2) * sizeof(float2);
}
size_t smem_y(const tdgl_sim *s, int cnt) { return 2ull * cnt * (s->My + 1) * sizeof(float2); }
size_t smem_z(const tdgl_sim *s, int cnt) { return 2ull * 3 * cnt * (s->Mz + 1) * sizeof(float2); }

int upload_items(tdgl_sim *s) {
    tdgl_ctx *ctx = s->ctx;
    cudaFree(s->d_rows); cudaFree(s->d_y); cudaFree(s->d_z);
    s->d_rows = s->d_y = s->d_z = nullptr;
    CK(ctx, cudaMalloc(&s->d_rows, s->it_rows.size() * sizeof(int4)));
    CK(ctx, cudaMemcpy(s->d_rows, s->it_rows.data(), s->it_rows.size() * sizeof(int4), cudaMemcpyHostToDevice));
    CK(ctx, cudaMalloc(&s->d_y, s->it_y.size() * sizeof(int4)));
    CK(ctx, cudaMemcpy(s->d_y, s->it_y.data(), s->it_y.size() * sizeof(int4), cudaMemcpyHostToDevice));
    CK(ctx, cudaMalloc(&s->d_z, s->it_z.size() * sizeof(int4)));
    CK(ctx, cudaMemcpy(s->d_z, s->it_z.data(), s->it_z.size() * sizeof(int4), cudaMemcpyHostToDevice));
    return TDGL_OK;
}

// -- normalization and coefficient table --------------------------------------------------------
int lowest_material(const tdgl_sim *s) {
    for (int i = 1; i < TDGL_MAX_MATERIALS; ++i)
        if (s->defined[i]) return i;
    return 0;
}

void fix_scales(tdgl_sim *s) {
    if (s->scales_fixed) return;
    const int m = lowest_material(s);
    double a = m ? fabs(alpha1_of(s->mats[m], 300.0)) : 0.0;
    if (!(a > 0.0) || !std::isfinite(a)) a = 1e8;
    double p = m ? tetragonal_ps(s->mats[m], 300.0) : 0.0;
    if (!(p > 0.0) || !std::isfinite(p)) p = 1.0;
    s->alpha_ref = a;
    s->P0 = p;
    s->scales_fixed = true;
}

void coef_table(const tdgl_sim *s, float *tab) {
    memset(tab, 0, sizeof(float) * MAXMAT * NCOEF);
    const double a = s->alpha_ref, P0 = s->P0, l2 = s->ell * s->ell, T = s->T;
    for (int id = 1; id < TDGL_MAX_MATERIALS; ++id) {
        if (!s->defined[id]) continue;
        const tdgl_material &m = s->mats[id];
        const double a1 = alpha1_of(m, T);
        const double a11 = m.a11_0 + m.a11_T * (T - m.a11_Tref);
        const double a111 = m.a111_0 + m.a111_T * (T - m.a111_Tref);
        float *c = tab + id * NCOEF;
        c[0] = (float)(a1 / a);
        c[1] = (float)(a1 / a);
        c[2] = (float)(m.r_s * a1 / a);
        c[3] = (float)(a11 * P0 * P0 / a);
        c[4] = (float)(m.a12 * P0 * P0 / a);
        c[5] = (float)(a111 * P0 * P0 * P0 * P0 / a);
        c[6] = (float)(m.a112 * P0 * P0 * P0 * P0 / a);
        c[7] = (float)(m.a123 * P0 * P0 * P0 * P0 / a);
        c[8] = (float)(m.G11 / (a * l2));
        c[9] = (float)((m.G44 + m.G44p) / (a * l2));
        c[10] = (float)(m.G12 / (a * l2));
        c[11] = (float)((m.G44 - m.G44p) / (a * l2));
    }
}

bool any_cross(const tdgl_sim *s) {
    for (int id = 1; id < TDGL_MAX_MATERIALS; ++id)
        if (s->defined[id] && (s->mats[id].G12 != 0.0 || s->mats[id].G44 != s->mats[id].G44p)) return true;
    return false;
}

// -- tensor spectrum -----------------------------------------------------------------------------
void gauss_legendre01(int m, double *tau, double *wt) {
    // m-point Gauss-Legendre on [0, 1] (Newton on the Legendre recurrence), weights times (1 - tau)
    for (int i = 0; i < m; ++i) {
        double x = cos(M_PI * (i + 0.75) / (m + 0.5)), dp = 1.0;
        for (int it = 0; it < 60; ++it) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= m; ++k) {
                const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = m * (x * p1 - p0) / (x * x - 1.0);
            const double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-15) break;
        }
        double p0 = 1.0, p1 = x;
        for (int k = 2; k <= m; ++k) {
            const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = m * (x * p1 - p0) / (x * x - 1.0);
        const double w = 2.0 / ((1.0 - x * x) * dp * dp);
        tau[i] = 0.5 * (1.0 + x);
        wt[i] = 0.5 * w * (1.0 - tau[i]);
    }
}

int build_tensor(tdgl_sim *s) {
    tdgl_ctx *ctx = s->ctx;
    const int nx = s->nx, ny = s->ny, nz = s->nz;
    FarRule rule;
    memset(&rule, 0, sizeof rule);
    const int ms[3] = {8, 6, 4};
    for (int q = 0; q < 3; ++q) {
        rule.m[q] = ms[q];
        gauss_legendre01(ms[q], rule.tau[q], rule.wt[q]);
    }
    const double l = s->ell;
    double *dN = nullptr, *dT1 = nullptr, *dT2 = nullptr, *dtrig = nullptr;
    const long nreal = (long)nx * ny * nz;
    const long n1 = (long)nz * ny * s->Kx, n2 = (long)nz * s->kyh * s->Kx, n3 = (long)s->kzh * s->kyh * s->Kx;
    CK(ctx, cudaMalloc(&dN, 6 * nreal * sizeof(double)));
    CK(ctx, cudaMalloc(&dT1, 6 * std::max(n1, n3) * sizeof(double)));   // passes x and z write here
    CK(ctx, cudaMalloc(&dT2, 6 * std::max(n2, n3) * sizeof(double)));
    const int Ms[3] = {s->Mx, s->My, s->Mz};
    std::vector<double> trig;
    size_t off[3];
    for (int a = 0; a < 3; ++a) {
        off[a] = trig.size();
        for (int t = 0; t < Ms[a]; ++t) trig.push_back(cos(2.0 * M_PI * t / Ms[a]));
        for (int t = 0; t < Ms[a]; ++t) trig.push_back(sin(2.0 * M_PI * t / Ms[a]));
    }
    CK(ctx, cudaMalloc(&dtrig, trig.size() * sizeof(double)));
    CK(ctx, cudaMemcpyAsync(dtrig, trig.data(), trig.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    // lengths in units of the smallest cell edge
    TRY(launch(ctx, TDGL_K_OTHER, [&] {
        k_tensor_real<<<grid_for(nreal), 256, 0, ctx->stream>>>(dN, nx, ny, nz, s->d[0] / l, s->d[1] / l, s->d[2] / l,
                                                                  5.0, 16.0, 40.0, rule);
    }));
    TRY(launch(ctx, TDGL_K_OTHER, [&] {
        k_tensor_dft<<<grid_for(6 * n1), 256, 0, ctx->stream>>>(dN, dT1, 0, nx, s->Kx, s->Mx, 1, nz * ny,
                                                                  dtrig + off[0], dtrig + off[0] + s->Mx);
    }));
    TRY(launch(ctx, TDGL_K_OTHER, [&] {
        k_tensor_dft<<<grid_for(6 * n2), 256, 0, ctx->stream>>>(dT1, dT2, 1, ny, s->kyh, s->My, s->Kx, nz,
                                                                  dtrig + off[1], dtrig + off[1] + s->My);
    }));
    TRY(launch(ctx, TDGL_K_OTHER, [&] {
        k_tensor_dft<<<grid_for(6 * n3), 256, 0, ctx->stream>>>(dT2, dT1, 2, nz, s->kzh, s->Mz, s->kyh * s->Kx, 1,
                                                                  dtrig + off[2], dtrig + off[2] + s->Mz);
    }));
    TRY(launch(ctx, TDGL_K_OTHER, [&] {
        k_tensor_store<<<grid_for(3L * s->kzh * s->kyh * s->kxp), 256, 0, ctx->stream>>>(dT1, s->dNhat, (long)s->kzh * s->kyh,
                                                                                         s->Kx, s->kxp);
    }));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    cudaFree(dN);
    cudaFree(dT1);
    cudaFree(dT2);
    cudaFree(dtrig);
    s->tensor_ready = true;
    return TDGL_OK;
}

int alloc_spectra(tdgl_sim *s) {
    if (s->spectra_alloc) return TDGL_OK;
    tdgl_ctx *ctx = s->ctx;
    CK(ctx, cudaMalloc(&s->dX, 3ull * s->nz * s->ny * s->kxp * sizeof(float2)));
    CK(ctx, cudaMalloc(&s->dY, 3ull * s->nz * s->My * s->kxp * sizeof(float2)));
    CK(ctx, cudaMalloc(&s->dNhat, 3ull * s->kzh * s->kyh * s->kxp * sizeof(float2)));
    s->spectra_alloc = true;
    // the z pass's TMA view of Y: float32 (2 kxp, My, nz, 3), box (2 KX, 1, nz, 1) where KX is the
    // pass's lines per block (the same for both radix-schedule variants)
    s->has_ymap = s->has_nmap = false;
    if (s->zN && s->nz <= 256) {
        auto enc = tmap_encode();
        const int KX = fast_zlines(s->Mz);
        const cuuint64_t dims[4] = {2ull * s->kxp, (cuuint64_t)s->My, (cuuint64_t)s->nz, 3};
        const cuuint64_t strides[3] = {8ull * s->kxp, 8ull * s->kxp * s->My, 8ull * s->kxp * s->My * s->nz};
        const cuuint32_t box[4] = {(cuuint32_t)(2 * KX), 1, (cuuint32_t)s->nz, 1};
        const cuuint32_t es[4] = {1, 1, 1, 1};
        s->has_ymap = enc && enc(&s->ymap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, s->dY, dims, strides, box, es,
                                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                 CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
        // the staged variant's view of the tensor table: float32 (2 kxp, kyh, kzh, 3), box
        // (2 KX, 1, kzh, 1), all kz rows of one reduced ky and KX columns per copy
        const cuuint64_t ndims[4] = {2ull * s->kxp, (cuuint64_t)s->kyh, (cuuint64_t)s->kzh, 3};
        const cuuint64_t nstrides[3] = {8ull * s->kxp, 8ull * s->kxp * s->kyh, 8ull * s->kxp * s->kyh * s->kzh};
        const cuuint32_t nbox[4] = {(cuuint32_t)(2 * KX), 1, (cuuint32_t)s->kzh, 1};
        s->has_nmap = s->has_ymap && s->kzh <= 256 &&
                      enc(&s->nmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, s->dNhat, ndims, nstrides, nbox, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    }
    return TDGL_OK;
}

// rebuild the device descriptor; P[0] is the current buffer
void fill_desc(tdgl_sim *s, double dt, unsigned terms) {
    SimDev &D = s->desc;
    memset(&D, 0, sizeof D);
    D.nx = s->nx; D.ny = s->ny; D.nz = s->nz; D.ncell = s->ncell;
    D.hx = s->hx; D.Kx = s->Kx; D.kxp = s->kxp; D.My = s->My; D.Mz = s->Mz; D.kyh = s->kyh; D.kzh = s->kzh;
    D.px = s->px; D.py = s->py; D.pz = s->pz; D.twr = s->twr; D.tw = s->dtw;
    D.P[0] = s->dP[s->cur]; D.P[1] = s->dP[s->cur ^ 1];
    D.mat = s->dmat; D.X = s->dX; D.Y = s->dY; D.Nhat = s->dNhat; D.coef = s->dcoef;
    for (int a = 0; a < 3; ++a) {
        const double h = s->d[a] / s->ell;
        D.inv_d2[a] = (float)(1.0 / (h * h));
        D.inv_2d[a] = (float)(1.0 / (2.0 * h));
        D.eext[a] = (float)(s->E[a] / (s->alpha_ref * s->P0));
        D.eac[a] = (float)(s->Eac[a] / (s->alpha_ref * s->P0));
    }
    D.ac_ph0 = 2.0 * M_PI * s->ac_freq * s->time + s->ac_phase;
    // phase per unit of the launch index: Euler step i uses index i; Heun's predictor and
    // corrector of step i use 2i and 2i + 2 (times t_i and t_i + dt)
    D.ac_dph = 2.0 * M_PI * s->ac_freq * dt / (s->integrator == TDGL_HEUN ? 2.0 : 1.0);
    D.hbuf = s->dhbuf;
    D.dt = (float)(s->alpha_ref * dt);
    D.escale = (float)(-1.0 / (kEps0 * s->eps_b * s->alpha_ref) / ((double)s->Mx * s->My * s->Mz));
    D.pmax = 1e3f;
    D.terms = terms;
    D.has_cross = s->has_cross ? 1 : 0;
    D.maxdp = s->dmaxdp; D.flag = s->dflag; D.energy = s->denergy;
    D.out = s->dout;
    D.out_scale = (float)(s->alpha_ref * s->P0);
    D.has_ymap = s->has_ymap ? 1 : 0;
    if (s->has_ymap) D.ymap = s->ymap;
    D.has_nmap = s->has_nmap ? 1 : 0;
    if (s->has_nmap) D.nmap = s->nmap;
}

int autotune_z(tdgl_sim *s);
int autotune_rows(tdgl_sim *s);

int prepare(tdgl_sim *s, unsigned need_terms) {
    tdgl_ctx *ctx = s->ctx;
    if (s->dirty) {   // validation and coefficient upload only after a change
        for (size_t i = 0; i < s->map.size(); ++i)
            if (s->map[i] && !s->defined[s->map[i]])
                return fail(ctx, TDGL_ESTATE, "material id %d used in the map but not defined", (int)s->map[i]);
        if (!lowest_material(s)) return fail(ctx, TDGL_ESTATE, "no material defined");
        fix_scales(s);
        s->has_cross = any_cross(s);
        float tab[MAXMAT * NCOEF];
        coef_table(s, tab);
        CK(ctx, cudaMemcpyAsync(s->dcoef, tab, sizeof tab, cudaMemcpyHostToDevice, ctx->stream));
        s->dirty = false;
    }
    if (need_terms & TDGL_TERM_ELEC) {
        TRY(alloc_spectra(s));
        if (!s->tensor_ready) TRY(build_tensor(s));
        TRY(autotune_z(s));
    }
    TRY(autotune_rows(s));
    return TDGL_OK;
}

int upload_desc(tdgl_sim *s) {
    CK(s->ctx, cudaMemcpyAsync(s->ddesc, &s->desc, sizeof(SimDev), cudaMemcpyHostToDevice, s->ctx->stream));
    return TDGL_OK;
}

// -- kernel sequences (over a descriptor table and item lists) ---------------------------------------
struct Group {
    int N;              // specialized transform length, 0 = generic kernel; for row groups -N marks
                        // rows shorter than the x half-length N (the step kernel's SHORT form)
    const int4 *items;
    int n;
    size_t smem;        // dynamic shared memory (generic kernels only)
};

// row-group length of a sim: its x half-length, negative when its rows are shorter (SHORT kernel)
int row_group_len(const tdgl_sim *s) { return (s->xN && s->nx < s->xN) ? -s->xN : s->xN; }

struct Work {
    const SimDev *descs;
    std::vector<Group> rg, yg, zg;   // row, y and z work by transform length
};

template <int MODE>
void rows_launch(const Group &g, const SimDev *d, cudaStream_t st, int parity) {
    if (g.N == 0) {
        k_rows<MODE><<<g.n, NTHREADS, g.smem, st>>>(d, g.items, parity);
        return;
    }
    const bool sh = g.N < 0;
    switch (sh ? -g.N : g.N) {
#define TDGL_R(LEN)                                                                               \
    case LEN:                                                                                     \
        if (sh) k_xrows<MODE, LEN, true><<<g.n, xrows_threads<LEN>(), g.smem, st>>>(d, g.items, parity); \
        else k_xrows<MODE, LEN><<<g.n, xrows_threads<LEN>(), g.smem, st>>>(d, g.items, parity);   \
        break;
        TDGL_FAST_LENGTHS(TDGL_R)
#undef TDGL_R
    }
}

int launch_rows(tdgl_ctx *ctx, int mode, const Work &w, int parity) {
    const int kind = (mode == MODE_XFWD) ? TDGL_K_XFWD : (mode_updates(mode) ? TDGL_K_STEP : TDGL_K_OTHER);
    for (const Group &g : w.rg) {
        if (g.n == 0) continue;
        TRY(launch(ctx, kind, [&] {
            switch (mode) {
                case MODE_STEP: rows_launch<MODE_STEP>(g, w.descs, ctx->stream, parity); break;
                case MODE_HEUN1: rows_launch<MODE_HEUN1>(g, w.descs, ctx->stream, parity); break;
                case MODE_HEUN2: rows_launch<MODE_HEUN2>(g, w.descs, ctx->stream, parity); break;
                case MODE_FIELD: rows_launch<MODE_FIELD>(g, w.descs, ctx->stream, parity); break;
                case MODE_DERIV: rows_launch<MODE_DERIV>(g, w.descs, ctx->stream, parity); break;
                case MODE_ENERGY: rows_launch<MODE_ENERGY>(g, w.descs, ctx->stream, parity); break;
                default: rows_launch<MODE_XFWD>(g, w.descs, ctx->stream, parity); break;
            }
        }));
    }
    return TDGL_OK;
}

template <bool INV>
void ypass(const Group &g, const SimDev *d, cudaStream_t st) {
    if (g.N == 0) {
        if (INV) k_yinv<<<g.n, NTHREADS, g.smem, st>>>(d, g.items);
        else k_yfwd<<<g.n, NTHREADS, g.smem, st>>>(d, g.items);
        return;
    }
    switch (g.N) {
#define TDGL_Y(LEN) \
    case LEN: k_ypass<LEN, INV><<<g.n, rf::threads_per_line<LEN>() * lines_per_block<LEN>(), 0, st>>>(d, g.items); break;
        TDGL_FAST_LENGTHS(TDGL_Y)
#undef TDGL_Y
    }
}

int zvar_index(int N) { return N == 256 ? 0 : (N == 512 ? 1 : (N == 128 ? 2 : -1)); }
// radix-schedule variants of the z pass per length: 128 and 256 have four (V = 2 stages the tensor
// rows, V = 3 also transforms the three components together), 512 two (its staged tile would not
// fit beside the spectra)
int zvar_count(int N) { return (N == 128 || N == 256) ? 4 : (N == 512 ? 2 : 0); }

template <int N, int V>
void zpass_v(const Group &g, const SimDev *d, cudaStream_t st) {
    if constexpr (V == 3)
        k_zpass3<N><<<g.n, ZCfg<N, V>::T * zlines_per_block<N, V>(), zpass_smem<N, V>(), st>>>(d, g.items);
    else
        k_zpass<N, V><<<g.n, ZCfg<N, V>::T * zlines_per_block<N, V>(), zpass_smem<N, V>(), st>>>(d, g.items);
}

// variant v of the z pass for LEN-point lines (a template, so the lengths without variants
// instantiate only variant 0)
template <int LEN> void zpass_len(int v, const Group &g, const SimDev *d, cudaStream_t st) {
    if constexpr (LEN == 128 || LEN == 256) {
        if (v == 3) zpass_v<LEN, 3>(g, d, st);
        else if (v == 2) zpass_v<LEN, 2>(g, d, st);
        else if (v == 1) zpass_v<LEN, 1>(g, d, st);
        else zpass_v<LEN, 0>(g, d, st);
    } else if constexpr (LEN == 512) {
        if (v == 1) zpass_v<LEN, 1>(g, d, st);
        else zpass_v<LEN, 0>(g, d, st);
    } else {
        zpass_v<LEN, 0>(g, d, st);
    }
}
template <int LEN> void zpass_attrs(int smem) {
    cudaFuncSetAttribute(k_zpass<LEN, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if constexpr (LEN == 128 || LEN == 256 || LEN == 512)
        cudaFuncSetAttribute(k_zpass<LEN, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if constexpr (LEN == 128 || LEN == 256) {
        cudaFuncSetAttribute(k_zpass<LEN, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        cudaFuncSetAttribute(k_zpass3<LEN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    }
}

// the z pass of one group with the context's radix-schedule variant (forced >= 0, else tuned)
void zpass(tdgl_ctx *ctx, const Group &g, const SimDev *d, int force = -1) {
    cudaStream_t st = ctx->stream;
    if (g.N == 0) {
        k_zconv<<<g.n, NTHREADS, g.smem, st>>>(d, g.items);
        return;
    }
    const int vi = zvar_index(g.N);
    const int v = force >= 0 ? force : ((vi >= 0 && ctx->zvar[vi] > 0) ? ctx->zvar[vi] : 0);
    switch (g.N) {
#define TDGL_Z(LEN)                   \
    case LEN:                         \
        zpass_len<LEN>(v, g, d, st);  \
        break;
        TDGL_FAST_LENGTHS(TDGL_Z)
#undef TDGL_Z
    }
}

int launch_conv(tdgl_ctx *ctx, const Work &w) {
    for (const Group &g : w.yg) TRY(launch(ctx, TDGL_K_YFWD, [&] { ypass<false>(g, w.descs, ctx->stream); }));
    for (const Group &g : w.zg) TRY(launch(ctx, TDGL_K_ZCONV, [&] { zpass(ctx, g, w.descs); }));
    for (const Group &g : w.yg) TRY(launch(ctx, TDGL_K_YINV, [&] { ypass<true>(g, w.descs, ctx->stream); }));
    return TDGL_OK;
}

Work sim_work(tdgl_sim *s, bool elec) {
    Work w;
    w.descs = s->ddesc;
    w.rg.push_back(Group{row_group_len(s), s->d_rows, (int)s->it_rows.size(), smem_rows(s, s->rows_cnt_max)});
    if (elec) {
        w.yg.push_back(Group{s->yN, s->d_y, (int)s->it_y.size(), s->yN ? 0 : smem_y(s, s->ky_cnt_max)});
        w.zg.push_back(Group{s->zN, s->d_z, (int)s->it_z.size(), s->zN ? 0 : smem_z(s, s->kz_cnt_max)});
    }
    return w;
}

// Radix-schedule autotuner of the z pass: the first time a context meets 256- or 512-point z
// lines, every variant of that length runs on this sim's own buffers (one launch to warm up,
// three timed with CUDA events) and the fastest is kept for the context.  The z pass works in place on the
// y-padded spectrum, which the next y pass rewrites, so the trial launches change no state.
int autotune_z(tdgl_sim *s) {
    tdgl_ctx *ctx = s->ctx;
    const int vi = zvar_index(s->zN);
    if (vi < 0 || ctx->zvar[vi] >= 0) return TDGL_OK;
    fill_desc(s, 0.0, s->terms);
    TRY(upload_desc(s));
    Work w = sim_work(s, true);
    const Group &g = w.zg[0];
    cudaEvent_t e0, e1;
    CK(ctx, cudaEventCreate(&e0));
    CK(ctx, cudaEventCreate(&e1));
    double us[kZVariants] = {0.0};
    const int nv = zvar_count(s->zN);
    for (int v = 0; v < nv; ++v) {
        TRY(launch(ctx, TDGL_K_OTHER, [&] { zpass(ctx, g, w.descs, v); }));
        CK(ctx, cudaEventRecord(e0, ctx->stream));
        for (int r = 0; r < 3; ++r) TRY(launch(ctx, TDGL_K_OTHER, [&] { zpass(ctx, g, w.descs, v); }));
        CK(ctx, cudaEventRecord(e1, ctx->stream));
        CK(ctx, cudaEventSynchronize(e1));
        float ms = 0.f;
        CK(ctx, cudaEventElapsedTime(&ms, e0, e1));
        us[v] = 1e3 * ms / 3.0;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int best = 0;
    for (int v = 0; v < kZVariants; ++v) {
        ctx->zus[vi][v] = us[v];
        if (v < nv && us[v] < us[best]) best = v;
    }
    ctx->zvar[vi] = best;
    return TDGL_OK;
}

// Row-tile autotuner (sims run alone): each candidate tile height runs the step kernel on scratch
// copies of the x-spectrum and of the P buffer it writes (and on scratch status slots), so the
// trial launches change no state; one launch warms up, three are timed with CUDA events.  The
// choice is kept per (x half-length, ny, nz, electrostatics) in the context.  Runs before the sim
// has captured any graph (its first preparation), since it rebuilds the sim's row items.
int autotune_rows(tdgl_sim *s) {
    if (s->rows_tuned) return TDGL_OK;
    tdgl_ctx *ctx = s->ctx;
    const int elec = (s->terms & TDGL_TERM_ELEC) ? 1 : 0;
    if (elec && !s->spectra_alloc) return TDGL_OK;   // tuned once the spectra exist
    s->rows_tuned = true;
    if (!s->xN || ctx->profiling || !s->d_rows) return TDGL_OK;
    for (const auto &r : ctx->rowtune)
        if (r.hx == s->hx && r.ny == s->ny && r.nz == s->nz && r.elec == elec) {
            s->row_tile = r.tile;
            memcpy(s->row_cand, r.cand, sizeof r.cand);
            memcpy(s->row_us, r.us, sizeof r.us);
            build_items(s);
            return upload_items(s);
        }
    // candidates: the kernel's tile, its half and quarter, the one-block-per-SM height
    const int full = s->rows_cnt_max;
    const long rows = (long)s->ny * s->nz;
    const int spread = (int)std::min<long>(full, std::max<long>(1, (rows + ctx->nsm - 1) / ctx->nsm));
    int cand[TDGL_ROW_CANDIDATES] = {0};
    int nc = 0;
    for (int c : {full, full / 2, full / 4, spread}) {
        bool seen = c < 1;
        for (int i = 0; i < nc; ++i) seen = seen || cand[i] == c;
        if (!seen && nc < TDGL_ROW_CANDIDATES) cand[nc++] = c;
    }
    double us[TDGL_ROW_CANDIDATES] = {0.0};
    float2 *xs = nullptr;
    float *ps = nullptr;
    unsigned *slots = nullptr;
    int4 *items = nullptr;
    SimDev *dd = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = TDGL_OK;
    auto ck = [&](cudaError_t e) {
        if (e != cudaSuccess && rc == TDGL_OK)
            rc = fail(ctx, e == cudaErrorMemoryAllocation ? TDGL_ENOMEM : TDGL_ECUDA, "row tuner: %s", cudaGetErrorString(e));
        return rc == TDGL_OK;
    };
    const size_t xbytes = elec ? 3ull * s->nz * s->ny * s->kxp * sizeof(float2) : 0;
    if (elec) ck(cudaMalloc(&xs, xbytes)) && ck(cudaMemcpyAsync(xs, s->dX, xbytes, cudaMemcpyDeviceToDevice, ctx->stream));
    ck(cudaMalloc(&ps, 3ull * s->ncell * sizeof(float))) && ck(cudaMalloc(&slots, 64)) &&
        ck(cudaMemsetAsync(slots, 0, 64, ctx->stream)) && ck(cudaMalloc(&dd, sizeof(SimDev))) &&
        ck(cudaMalloc(&items, ((rows + 0) * sizeof(int4)))) && ck(cudaEventCreate(&e0)) && ck(cudaEventCreate(&e1));
    if (rc == TDGL_OK) {
        fill_desc(s, 0.0, s->terms);
        SimDev D = s->desc;
        if (elec) D.X = xs;
        D.P[1] = ps;
        D.maxdp = slots;
        D.flag = reinterpret_cast<int *>(slots + 4);
        ck(cudaMemcpyAsync(dd, &D, sizeof D, cudaMemcpyHostToDevice, ctx->stream));
    }
    for (int c = 0; c < nc && rc == TDGL_OK; ++c) {
        std::vector<int4> it;
        for (int z = 0; z < s->nz; ++z)
            for (int y0 = 0; y0 < s->ny; y0 += cand[c]) it.push_back(make_int4(0, z, y0, std::min(cand[c], s->ny - y0)));
        if (!ck(cudaMemcpyAsync(items, it.data(), it.size() * sizeof(int4), cudaMemcpyHostToDevice, ctx->stream))) break;
        const Group g{row_group_len(s), items, (int)it.size(), smem_rows(s, s->rows_cnt_max)};
        rows_launch<MODE_STEP>(g, dd, ctx->stream, 0);
        ck(cudaEventRecord(e0, ctx->stream));
        for (int r = 0; r < 3; ++r) rows_launch<MODE_STEP>(g, dd, ctx->stream, 0);
        ck(cudaEventRecord(e1, ctx->stream));
        ck(cudaGetLastError());
        if (ck(cudaEventSynchronize(e1))) {
            float ms = 0.f;
            ck(cudaEventElapsedTime(&ms, e0, e1));
            us[c] = 1e3 * ms / 3.0;
        }
    }
    cudaStreamSynchronize(ctx->stream);
    cudaFree(xs);
    cudaFree(ps);
    cudaFree(slots);
    cudaFree(items);
    cudaFree(dd);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (rc != TDGL_OK) return rc;
    int best = 0;
    for (int c = 1; c < nc; ++c)
        if (us[c] < us[best]) best = c;
    tdgl_ctx::RowTune r{s->hx, s->ny, s->nz, elec, cand[best], {0}, {0.0}};
    memcpy(r.cand, cand, sizeof cand);
    memcpy(r.us, us, sizeof us);
    ctx->rowtune.push_back(r);
    s->row_tile = cand[best];
    memcpy(s->row_cand, cand, sizeof cand);
    memcpy(s->row_us, us, sizeof us);
    build_items(s);
    return upload_items(s);
}

// bring X to the E-hat state of the current P (descriptor already uploaded with P[0] = current)
int ensure_ehat(tdgl_sim *s, const Work &w) {
    if (s->xstate == XS_NONE) {
        TRY(launch_rows(s->ctx, MODE_XFWD, w, 0));
        s->xstate = XS_PHAT;
    }
    if (s->xstate == XS_PHAT) {
        TRY(launch_conv(s->ctx, w));
        s->xstate = XS_EHAT;
    }
    return TDGL_OK;
}

int read_status(tdgl_sim *s, double *maxdp, int *flag) {
    unsigned u = 0;
    int f = 0;
    CK(s->ctx, cudaMemcpyAsync(&u, s->dmaxdp, sizeof u, cudaMemcpyDeviceToHost, s->ctx->stream));
    CK(s->ctx, cudaMemcpyAsync(&f, s->dflag, sizeof f, cudaMemcpyDeviceToHost, s->ctx->stream));
    CK(s->ctx, cudaStreamSynchronize(s->ctx->stream));
    float v;
    memcpy(&v, &u, sizeof v);
    *maxdp = (u >= 0x7f800000u) ? INFINITY : (double)v;
    *flag = f;
    s->last_maxdp = *maxdp;
    return TDGL_OK;
}

// Launches of steps i0..n-1, starting from P-hat in X.  Euler: convolution, row kernel (launch
// index i, parity i & 1).  Heun: predictor on P (index 2i), convolution of the predictor,
// corrector (index 2i + 2); P stays in the same buffer.  maxdp is reset before the last step.
int record_steps(tdgl_sim *s, const Work &w, int i0, int n, bool elec, bool heun) {
    tdgl_ctx *ctx = s->ctx;
    for (int i = i0; i < n; ++i) {
        if (elec) TRY(launch_conv(ctx, w));
        if (heun) {
            TRY(launch_rows(ctx, MODE_HEUN1, w, 2 * i));
            if (elec) TRY(launch_conv(ctx, w));
            if (i == n - 1) CK(ctx, cudaMemsetAsync(s->dmaxdp, 0, sizeof(unsigned), ctx->stream));
            TRY(launch_rows(ctx, MODE_HEUN2, w, 2 * i + 2));
        } else {
            if (i == n - 1) CK(ctx, cudaMemsetAsync(s->dmaxdp, 0, sizeof(unsigned), ctx->stream));
            TRY(launch_rows(ctx, MODE_STEP, w, i));
        }
    }
    return TDGL_OK;
}

// n <= kStepChunk steps of one sim without a status read; maxdp reset before the last step
int steps_chunk(tdgl_sim *s, int n, double dt) {
    tdgl_ctx *ctx = s->ctx;
    const bool elec = (s->terms & TDGL_TERM_ELEC) != 0;
    fill_desc(s, dt, s->terms);
    TRY(upload_desc(s));
    Work w = sim_work(s, elec);
    if (elec && s->xstate == XS_NONE) {
        TRY(launch_rows(ctx, MODE_XFWD, w, 0));
        s->xstate = XS_PHAT;
    }
    const bool heun = s->integrator == TDGL_HEUN;
    int i0 = 0;
    if (elec && s->xstate == XS_EHAT) {   // the first step reuses the field spectrum already in X
        if (n == 1) CK(ctx, cudaMemsetAsync(s->dmaxdp, 0, sizeof(unsigned), ctx->stream));
        if (heun) {
            TRY(launch_rows(ctx, MODE_HEUN1, w, 0));
            TRY(launch_conv(ctx, w));
            TRY(launch_rows(ctx, MODE_HEUN2, w, 2));
        } else {
            TRY(launch_rows(ctx, MODE_STEP, w, 0));
        }
        i0 = 1;
    }
    auto record = [&]() -> int { return record_steps(s, w, i0, n, elec, heun); };
    const int m = n - i0;
    // repeated sequences replay a captured graph (the descriptor, read by the kernels from device
    // memory, carries dt and the current P buffer); not while profiling
    if (m >= 2 && !ctx->profiling && ctx->stream) {
        tdgl_sim::GraphRec *G = nullptr;
        const int p0 = heun ? 0 : (i0 & 1);
        for (auto &g : s->graphs)
            if (g.n == m && g.elec == elec && g.p0 == p0 && g.integ == s->integrator) G = &g;
        if (!G) {
            tdgl_sim::GraphRec r{m, elec, p0, s->integrator, nullptr, 0};
            TRY(capture_graph(ctx, record, &r.exec, &r.kernels));
            s->graphs.push_back(r);
            G = &s->graphs.back();
        }
        CK(ctx, cudaGraphLaunch(G->exec, ctx->stream));
        ctx->launches += G->kernels;
    } else if (m > 0) {
        TRY(record());
    }
    if ((n & 1) && !heun) s->cur ^= 1;
    s->xstate = elec ? XS_PHAT : XS_NONE;
    s->time += n * dt;
    return TDGL_OK;
}

// n steps of one sim without a status read; maxdp reset before the last step.  A long call runs as
// chunks of kStepChunk steps (even, so the buffer parity repeats), each replaying the same cached
// graph with its descriptor refreshed (the applied field's phase at the chunk's first step): the
// graphs a sim keeps stay few and small whatever n is.
constexpr int kStepChunk = 64;
int steps_nosync(tdgl_sim *s, int n, double dt) {
    for (int done = 0; done < n;) {
        const int len = std::min(kStepChunk, n - done);
        TRY(steps_chunk(s, len, dt));
        done += len;
    }
    return TDGL_OK;
}

// ---- multi-stage integrators (RK45, AB3M2) -----------------------------------------------------
// Runge-Kutta-Fehlberg 4(5) (Fehlberg 1969): nodes c, stage matrix a, fourth- and fifth-order weights
const double kRkfC[6] = {0.0, 1.0 / 4.0, 3.0 / 8.0, 12.0 / 13.0, 1.0, 1.0 / 2.0};
const double kRkfA[6][5] = {{0, 0, 0, 0, 0},
                            {1.0 / 4.0, 0, 0, 0, 0},
                            {3.0 / 32.0, 9.0 / 32.0, 0, 0, 0},
                            {1932.0 / 2197.0, -7200.0 / 2197.0, 7296.0 / 2197.0, 0, 0},
                            {439.0 / 216.0, -8.0, 3680.0 / 513.0, -845.0 / 4104.0, 0},
                            {-8.0 / 27.0, 2.0, -3544.0 / 2565.0, 1859.0 / 4104.0, -11.0 / 40.0}};
const double kRkfB4[6] = {25.0 / 216.0, 0.0, 1408.0 / 2565.0, 2197.0 / 4104.0, -1.0 / 5.0, 0.0};
const double kRkfB5[6] = {16.0 / 135.0, 0.0, 6656.0 / 12825.0, 28561.0 / 56430.0, -9.0 / 50.0, 2.0 / 55.0};

// dP/dt (normalized field) of the state in P[parity] into dst, the applied field taken at time t
int eval_deriv(tdgl_sim *s, const Work &w, int parity, float *dst, double t, bool elec) {
    tdgl_ctx *ctx = s->ctx;
    s->desc.hbuf = dst;
    s->desc.ac_ph0 = 2.0 * M_PI * s->ac_freq * t + s->ac_phase;
    s->desc.ac_dph = 0.0;
    TRY(upload_desc(s));
    if (elec) {
        TRY(launch_rows(ctx, MODE_XFWD, w, parity));
        TRY(launch_conv(ctx, w));
    }
    return launch_rows(ctx, MODE_DERIV, w, parity);
}

// out = P + h sum_j c[j] K[j] (material cells); track: max |h sum_j d[j] K[j]| and max |out - P|
int combine(tdgl_sim *s, float *out, const float *P, int nk, const float *const *K, const double *c, int nd,
            const double *d, double h, bool track) {
    Combine q;
    memset(&q, 0, sizeof q);
    q.out = out;
    q.P = P;
    q.nk = nk;
    q.nd = nd;
    q.mat = s->dmat;
    q.ncell = s->ncell;
    for (int j = 0; j < nk; ++j) {
        q.K[j] = K[j];
        q.c[j] = (float)(h * c[j]);
    }
    for (int j = 0; j < nd; ++j) q.d[j] = (float)(h * d[j]);
    if (track) {
        q.errmax = s->derrmax;
        q.dpmax = s->dmaxdp;
        CK(s->ctx, cudaMemsetAsync(s->derrmax, 0, sizeof(unsigned), s->ctx->stream));
        CK(s->ctx, cudaMemsetAsync(s->dmaxdp, 0, sizeof(unsigned), s->ctx->stream));
    }
    return launch(s->ctx, TDGL_K_OTHER, [&] { k_combine<<<grid_for(3 * s->ncell), 256, 0, s->ctx->stream>>>(q); });
}

int read_err_dp(tdgl_sim *s, double *err, double *dp) {
    unsigned u[2] = {0, 0};
    CK(s->ctx, cudaMemcpyAsync(&u[0], s->derrmax, sizeof(unsigned), cudaMemcpyDeviceToHost, s->ctx->stream));
    CK(s->ctx, cudaMemcpyAsync(&u[1], s->dmaxdp, sizeof(unsigned), cudaMemcpyDeviceToHost, s->ctx->stream));
    CK(s->ctx, cudaStreamSynchronize(s->ctx->stream));
    float f[2];
    memcpy(f, u, sizeof f);
    *err = (u[0] >= 0x7f800000u) ? INFINITY : (double)f[0];
    *dp = (u[1] >= 0x7f800000u) ? INFINITY : (double)f[1];
    return TDGL_OK;
}

// one RKF45 attempt of dt from P[cur]: six evaluations, the fourth-order solution into P[cur ^ 1]
int rk45_attempt(tdgl_sim *s, const Work &w, double dt, bool elec, double *err, double *dp) {
    const double h = s->alpha_ref * dt;
    fill_desc(s, dt, s->terms);
    float *P = s->dP[s->cur], *Q = s->dP[s->cur ^ 1];
    const size_t n3 = 3ull * s->ncell;
    float *K[6];
    for (int i = 0; i < 6; ++i) K[i] = s->dstage + i * n3;
    for (int i = 0; i < 6; ++i) {
        int par = 0;
        if (i > 0) {
            TRY(combine(s, Q, P, i, K, kRkfA[i], 0, nullptr, h, false));
            par = 1;
        }
        TRY(eval_deriv(s, w, par, K[i], s->time + kRkfC[i] * dt, elec));
    }
    double e[6];
    for (int j = 0; j < 6; ++j) e[j] = kRkfB5[j] - kRkfB4[j];
    TRY(combine(s, Q, P, 6, K, kRkfB4, 6, e, h, true));
    return read_err_dp(s, err, dp);
}

// one AB3M2 (PECE) step of dt: predictor from the newest three evaluations, evaluation at the
// prediction, corrector, evaluation at the new state (the newest history entry of the next step)
int ab3m2_step(tdgl_sim *s, const Work &w, double dt, bool elec, double *dp) {
    const double h = s->alpha_ref * dt;
    const size_t n3 = 3ull * s->ncell;
    float *F[3] = {s->dstage, s->dstage + n3, s->dstage + 2 * n3}, *Fs = s->dstage + 3 * n3;
    fill_desc(s, dt, s->terms);
    float *P = s->dP[s->cur], *Q = s->dP[s->cur ^ 1];
    if (s->ab_hist == 0) {
        s->ab_ring = 0;
        TRY(eval_deriv(s, w, 0, F[0], s->time, elec));
        s->ab_hist = 1;
    }
    const int r = s->ab_ring;
    const float *hist[3] = {F[r], F[(r + 2) % 3], F[(r + 1) % 3]};   // f_n, f_{n-1}, f_{n-2}
    static const double p1[1] = {1.0}, p2[2] = {1.5, -0.5}, p3[3] = {23.0 / 12.0, -16.0 / 12.0, 5.0 / 12.0};
    const double *pc = s->ab_hist == 1 ? p1 : (s->ab_hist == 2 ? p2 : p3);
    TRY(combine(s, Q, P, s->ab_hist, hist, pc, 0, nullptr, h, false));
    TRY(eval_deriv(s, w, 1, Fs, s->time + dt, elec));
    const float *kc[3] = {Fs, hist[0], hist[1]};
    static const double c1[2] = {0.5, 0.5}, c2[3] = {5.0 / 12.0, 8.0 / 12.0, -1.0 / 12.0};
    TRY(combine(s, Q, P, s->ab_hist == 1 ? 2 : 3, kc, s->ab_hist == 1 ? c1 : c2, 0, nullptr, h, true));
    double err;
    TRY(read_err_dp(s, &err, dp));
    if (!std::isfinite(*dp)) return fail(s->ctx, TDGL_EDIVERGED, "P diverged (NaN or |P| > 1e3 P0)");
    s->cur ^= 1;
    s->time += dt;
    fill_desc(s, dt, s->terms);
    s->ab_ring = (r + 1) % 3;
    TRY(eval_deriv(s, w, 0, F[s->ab_ring], s->time, elec));
    s->ab_hist = std::min(s->ab_hist + 1, 3);
    return TDGL_OK;
}

// n accepted steps of RK45 or AB3M2; *scaled_dp: max|dP| / P0 of the last step times dt_ref / dt
int multistage_steps(tdgl_sim *s, long n, double dt_ref, double *scaled_dp) {
    tdgl_ctx *ctx = s->ctx;
    const bool elec = (s->terms & TDGL_TERM_ELEC) != 0;
    fill_desc(s, dt_ref, s->terms);
    TRY(upload_desc(s));
    Work w = sim_work(s, elec);
    for (long k = 0; k < n; ++k) {
        double dp = 0.0, dt = dt_ref;
        if (s->integrator == TDGL_AB3M2) {
            TRY(ab3m2_step(s, w, dt, elec, &dp));
        } else {
            const bool adapt = s->ad_tol > 0;
            if (adapt && s->dt_next > 0) dt = s->dt_next;
            for (int tries = 0;; ++tries) {
                double err;
                TRY(rk45_attempt(s, w, dt, elec, &err, &dp));
                if (!std::isfinite(err) || !std::isfinite(dp))
                    return fail(ctx, TDGL_EDIVERGED, "P diverged (NaN or |P| > 1e3 P0)");
                const bool at_min = adapt && s->ad_min > 0 && dt <= s->ad_min;
                if (!adapt || err <= s->ad_tol || at_min) {
                    if (adapt) {
                        double f = err > 0 ? 0.9 * pow(s->ad_tol / err, 0.2) : 5.0;
                        f = std::min(5.0, std::max(0.2, f));
                        double dn = dt * f;
                        if (s->ad_max > 0) dn = std::min(dn, s->ad_max);
                        if (s->ad_min > 0) dn = std::max(dn, s->ad_min);
                        s->dt_next = dn;
                    }
                    break;
                }
                if (tries >= 60) return fail(ctx, TDGL_ENOTCONVERGED, "RK45 step rejected 60 times (dt %g s)", dt);
                dt *= std::min(1.0, std::max(0.1, 0.9 * pow(s->ad_tol / err, 0.25)));
                if (s->ad_min > 0) dt = std::max(dt, s->ad_min);
            }
            s->cur ^= 1;
            s->time += dt;
        }
        s->last_maxdp = dp;
        *scaled_dp = dp * dt_ref / dt;
    }
    s->xstate = XS_NONE;
    return TDGL_OK;
}

bool valid_where(int w) { return w == TDGL_HOST || w == TDGL_DEVICE; }

int copy_in(tdgl_ctx *ctx, void *dst, const void *src, size_t bytes, int where) {
    CK(ctx, cudaMemcpyAsync(dst, src, bytes, where == TDGL_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                            ctx->stream));
    return TDGL_OK;
}

int copy_out(tdgl_ctx *ctx, void *dst, const void *src, size_t bytes, int where) {
    CK(ctx, cudaMemcpyAsync(dst, src, bytes, where == TDGL_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                            ctx->stream));
    if (where == TDGL_HOST) CK(ctx, cudaStreamSynchronize(ctx->stream));
    return TDGL_OK;
}

int ensure_out(tdgl_sim *s) {
    if (!s->dout) CK(s->ctx, cudaMalloc(&s->dout, 3ull * s->ncell * sizeof(float)));
    return TDGL_OK;
}

}  // namespace

// =============================================================================================
extern "C" {

int tdgl_ctx_create(tdgl_ctx **out, int device, void *stream) {
    if (!out) return TDGL_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return TDGL_ECUDA;
    tdgl_ctx *ctx = new tdgl_ctx();
    ctx->device = device;
    if (cudaSetDevice(device) != cudaSuccess) { delete ctx; return TDGL_ECUDA; }
    if (cudaDeviceGetAttribute(&ctx->nsm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || ctx->nsm < 1) {
        delete ctx;
        return TDGL_ECUDA;
    }
    if (stream) {
        ctx->stream = (cudaStream_t)stream;
    } else {
        if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) { delete ctx; return TDGL_ECUDA; }
        ctx->own_stream = true;
    }
    cudaFuncSetAttribute(k_rows<MODE_STEP>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
    cudaFuncSetAttribute(k_rows<MODE_FIELD>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
    cudaFuncSetAttribute(k_rows<MODE_ENERGY>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
    cudaFuncSetAttribute(k_rows<MODE_XFWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
    cudaFuncSetAttribute(k_rows<MODE_HEUN1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
    cudaFuncSetAttribute(k_rows<MODE_HEUN2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
    cudaFuncSetAttribute(k_rows<MODE_DERIV>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
    cudaFuncSetAttribute(k_yfwd, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
    cudaFuncSetAttribute(k_yinv, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
    cudaFuncSetAttribute(k_zconv, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
#define TDGL_XA(LEN)                                                                                    \
    cudaFuncSetAttribute(k_xrows<MODE_STEP, LEN>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);   \
    cudaFuncSetAttribute(k_xrows<MODE_FIELD, LEN>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);  \
    cudaFuncSetAttribute(k_xrows<MODE_ENERGY, LEN>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem); \
    cudaFuncSetAttribute(k_xrows<MODE_XFWD, LEN>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);   \
    cudaFuncSetAttribute(k_xrows<MODE_HEUN1, LEN>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);  \
    cudaFuncSetAttribute(k_xrows<MODE_HEUN2, LEN>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);  \
    cudaFuncSetAttribute(k_xrows<MODE_DERIV, LEN>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);  \
    cudaFuncSetAttribute(k_xrows<MODE_STEP, LEN, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);   \
    cudaFuncSetAttribute(k_xrows<MODE_FIELD, LEN, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);  \
    cudaFuncSetAttribute(k_xrows<MODE_ENERGY, LEN, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem); \
    cudaFuncSetAttribute(k_xrows<MODE_XFWD, LEN, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);   \
    cudaFuncSetAttribute(k_xrows<MODE_HEUN1, LEN, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);  \
    cudaFuncSetAttribute(k_xrows<MODE_HEUN2, LEN, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);  \
    cudaFuncSetAttribute(k_xrows<MODE_DERIV, LEN, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
    TDGL_FAST_LENGTHS(TDGL_XA)
#undef TDGL_XA
#define TDGL_ZA(LEN) zpass_attrs<LEN>(kMaxSmem);
    TDGL_FAST_LENGTHS(TDGL_ZA)
#undef TDGL_ZA
    if (cudaGetLastError() != cudaSuccess) { delete ctx; return TDGL_ECUDA; }
    *out = ctx;
    return TDGL_OK;
}

void tdgl_ctx_destroy(tdgl_ctx *ctx) {
    if (!ctx) return;
    ctx_set(ctx);
    cudaStreamSynchronize(ctx->stream);
    const std::vector<tdgl_batch *> bs = ctx->batches;
    for (auto b : bs) tdgl_batch_destroy(b);
    const std::vector<tdgl_sim *> ss = ctx->sims;
    for (auto sm : ss) tdgl_sim_destroy(sm);
    const std::vector<tdgl_unet *> ns = ctx->nets;
    for (auto n : ns) tdgl_unet_destroy(n);
    for (auto &r : ctx->recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto e : ctx->pool) cudaEventDestroy(e);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    cudaFree(ctx->splitk);
    if (ctx->up) cudaStreamDestroy(ctx->up);
    if (ctx->down) cudaStreamDestroy(ctx->down);
    delete ctx;
}

const char *tdgl_last_error(const tdgl_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }
long tdgl_launch_count(const tdgl_ctx *ctx) { return ctx ? ctx->launches : 0; }

// FP32 FMA throughput probe: 8 independent dependency chains per thread, so every SM sub-partition
// has independent FMAs to issue each cycle; the result is stored only if it equals a value it never
// takes, which keeps the chains from being removed
__global__ void __launch_bounds__(256) k_fma_peak(float *sink, int iters, float b, float c) {
    float a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = (float)(threadIdx.x + k) * 1e-3f;
#pragma unroll 8
    for (int i = 0; i < iters; ++i) {   // unrolled: loop control is a few instructions per 64 FMAs
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = fmaf(a[k], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    if (s == -1.2345f) sink[0] = s;
}

// Timeout probe: thread 0 waits for phase 0 of an mbarrier that expects one arrival nobody makes (no
// copy is in flight, so giving up leaves nothing outstanding), at most `polls` polls, and records
// the timeout in flag bit 1 as the pipelined kernels do.
__global__ void k_wait_probe(int *flag, long polls) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);
        tc::mbar_fence_init();
        if (!tc::mbar_wait(&bar, 0u, polls)) atomicOr(flag, 2);
    }
}

int tdgl_wait_probe(tdgl_ctx *ctx, long polls) {
    if (!ctx) return TDGL_EINVAL;
    if (polls < 1 || polls > (1L << 24)) return fail(ctx, TDGL_EINVAL, "poll count %ld", polls);
    ctx_set(ctx);
    int *dflag = nullptr;
    CK(ctx, cudaMalloc(&dflag, sizeof(int)));
    int h = 0;
    cudaError_t e = cudaMemsetAsync(dflag, 0, sizeof(int), ctx->stream);
    if (e == cudaSuccess) {
        k_wait_probe<<<1, 32, 0, ctx->stream>>>(dflag, polls);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, dflag, sizeof h, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaFree(dflag);
    if (e != cudaSuccess) return fail(ctx, TDGL_ECUDA, "wait probe: %s", cudaGetErrorString(e));
    ctx->launches++;
    if (h & 2) return fail(ctx, TDGL_ETIMEOUT, "the probe's bounded wait gave up after %ld polls", polls);
    return TDGL_OK;
}

int tdgl_fp32_fma_peak(tdgl_ctx *ctx, double *tflops) {
    if (!ctx || !tflops) return TDGL_EINVAL;
    ctx_set(ctx);
    float *sink = nullptr;
    CK(ctx, cudaMalloc(&sink, sizeof(float)));
    const int blocks = ctx->nsm * 8, threads = 256, iters = 1 << 14;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // b slightly below 1 and c small keep the chains finite
    k_fma_peak<<<blocks, threads, 0, ctx->stream>>>(sink, iters, 0.999999f, 1e-7f);
    cudaEventRecord(e0, ctx->stream);
    for (int r = 0; r < 3; ++r) k_fma_peak<<<blocks, threads, 0, ctx->stream>>>(sink, iters, 0.999999f, 1e-7f);
    cudaEventRecord(e1, ctx->stream);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    CK(ctx, e);
    CK(ctx, cudaGetLastError());
    const double flops = 2.0 * 8.0 * iters * (double)blocks * threads;
    *tflops = flops / (ms / 3.0 * 1e-3) / 1e12;
    return TDGL_OK;
}

// padded transform lengths of a sim: plans, the twiddle table (returned for upload) and work items
void set_lengths(tdgl_sim *s, int Mx, int My, int Mz, std::vector<float2> &tw) {
    s->Mx = Mx;
    s->My = My;
    s->Mz = Mz;
    s->hx = s->Mx / 2;
    s->Kx = s->hx + 1;
    s->kxp = (s->Kx + 3) & ~3;
    s->kyh = s->My / 2 + 1;
    s->kzh = s->Mz / 2 + 1;
    tw.clear();
    s->px = make_plan(s->hx, tw);
    s->py = make_plan(s->My, tw);
    s->pz = make_plan(s->Mz, tw);
    s->twr = (int)tw.size();
    for (int k = 0; k <= s->hx; ++k) {
        const double a = -2.0 * M_PI * (double)k / (double)s->Mx;
        tw.push_back(make_float2((float)cos(a), (float)sin(a)));
    }
    build_items(s);
}

int tdgl_sim_create(tdgl_ctx *ctx, int nx, int ny, int nz, double dx, double dy, double dz, tdgl_sim **out) {
    if (!ctx || !out) return TDGL_EINVAL;
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1 || nx > TDGL_MAX_DIM || ny > TDGL_MAX_DIM || nz > TDGL_MAX_DIM)
        return fail(ctx, TDGL_EINVAL, "grid %dx%dx%d outside 1..%d", nx, ny, nz, TDGL_MAX_DIM);
    if (!(dx > 0) || !(dy > 0) || !(dz > 0) || !std::isfinite(dx) || !std::isfinite(dy) || !std::isfinite(dz))
        return fail(ctx, TDGL_EINVAL, "cell sizes must be positive and finite");
    ctx_set(ctx);
    tdgl_sim *s = new tdgl_sim();
    s->ctx = ctx;
    s->nx = nx; s->ny = ny; s->nz = nz;
    s->d[0] = dx; s->d[1] = dy; s->d[2] = dz;
    s->ell = std::min(dx, std::min(dy, dz));
    s->ncell = (long)nx * ny * nz;
    memset(s->mats, 0, sizeof s->mats);
    s->map.assign(s->ncell, 0);
    std::vector<float2> tw;
    set_lengths(s, default_x_length(nx), default_y_length(ny), default_z_length(nz), tw);
    int rc = TDGL_OK;
    auto al = [&](void **p, size_t b) {
        if (rc != TDGL_OK) return;
        cudaError_t e = cudaMalloc(p, b);
        if (e != cudaSuccess) rc = fail(ctx, TDGL_ENOMEM, "cudaMalloc(%zu): %s", b, cudaGetErrorString(e));
    };
    al((void **)&s->dP[0], 3ull * s->ncell * sizeof(float));
    al((void **)&s->dP[1], 3ull * s->ncell * sizeof(float));
    al((void **)&s->dmat, s->ncell);
    al((void **)&s->dtw, tw.size() * sizeof(float2));
    al((void **)&s->dcoef, MAXMAT * NCOEF * sizeof(float));
    al((void **)&s->dmaxdp, sizeof(unsigned));
    al((void **)&s->dflag, sizeof(int));
    al((void **)&s->denergy, 4 * sizeof(double));
    al((void **)&s->ddesc, sizeof(SimDev));
    if (rc == TDGL_OK) {
        cudaMemsetAsync(s->dP[0], 0, 3ull * s->ncell * sizeof(float), ctx->stream);
        cudaMemsetAsync(s->dP[1], 0, 3ull * s->ncell * sizeof(float), ctx->stream);
        cudaMemsetAsync(s->dmat, 0, s->ncell, ctx->stream);
        cudaMemsetAsync(s->dflag, 0, sizeof(int), ctx->stream);
        cudaMemsetAsync(s->dmaxdp, 0, sizeof(unsigned), ctx->stream);
        cudaMemcpyAsync(s->dtw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice, ctx->stream);
        rc = upload_items(s);
        if (rc == TDGL_OK && cudaStreamSynchronize(ctx->stream) != cudaSuccess)
            rc = fail(ctx, TDGL_ECUDA, "sim setup: %s", cudaGetErrorString(cudaGetLastError()));
    }
    if (rc != TDGL_OK) {
        tdgl_sim_destroy(s);
        return rc;
    }
    ctx->sims.push_back(s);
    *out = s;
    return TDGL_OK;
}

void tdgl_sim_destroy(tdgl_sim *s) {
    if (!s) return;
    ctx_set(s->ctx);
    cudaStreamSynchronize(s->ctx->stream);
    for (int i = 0; i < 2; ++i) {
        if (s->ev_out_free[i]) cudaEventSynchronize(s->ev_out_free[i]);   // a download still reading dout_a
        for (cudaEvent_t e : {s->ev_in_ready[i], s->ev_in_free[i], s->ev_out_ready[i], s->ev_out_free[i]})
            if (e) cudaEventDestroy(e);
        cudaFree(s->din_a[i]);
        cudaFree(s->dout_a[i]);
    }
    auto &v = s->ctx->sims;
    v.erase(std::remove(v.begin(), v.end(), s), v.end());
    if (s->batch) {   // leave the batch rather than dangle in it
        auto &bv = s->batch->sims;
        bv.erase(std::remove(bv.begin(), bv.end(), s), bv.end());
        drop_cache(s->batch);              // indices in the cached work lists changed
    }
    for (auto &g : s->graphs) cudaGraphExecDestroy(g.exec);
    for (auto &g : s->relax_graphs) cudaGraphExecDestroy(g.exec);
    void *ptrs[] = {s->dP[0], s->dP[1], s->dmat, s->dX, s->dY, s->dNhat, s->dtw, s->dcoef, s->dmaxdp,
                    s->dflag, s->denergy, s->dout, s->ddesc, s->d_rows, s->d_y, s->d_z, s->dhbuf,
                    s->dstage, s->derrmax, s->drelax};
    for (void *p : ptrs) cudaFree(p);
    delete s;
}

int tdgl_material_define(tdgl_sim *s, int id, const tdgl_material *m) {
    if (!s || !m) return TDGL_EINVAL;
    if (id < 1 || id >= TDGL_MAX_MATERIALS) return fail(s->ctx, TDGL_EINVAL, "material id %d outside 1..%d", id, TDGL_MAX_MATERIALS - 1);
    if (m->a1_form < 0 || m->a1_form > 2) return fail(s->ctx, TDGL_EINVAL, "a1_form %d", m->a1_form);
    if (m->a1_form == 1 && (m->coth_Ts == 0.0 || m->coth_T1 <= 0.0)) return fail(s->ctx, TDGL_EINVAL, "coth form needs Ts != 0, T1 > 0");
    s->mats[id] = *m;
    s->defined[id] = true;
    s->dirty = true;
    return TDGL_OK;
}

static int apply_map(tdgl_sim *s) {
    tdgl_ctx *ctx = s->ctx;
    s->dirty = true;
    ctx_set(ctx);
    CK(ctx, cudaMemcpyAsync(s->dmat, s->map.data(), s->ncell, cudaMemcpyHostToDevice, ctx->stream));
    TRY(launch(ctx, TDGL_K_OTHER, [&] { k_mask<<<grid_for(3 * s->ncell), 256, 0, ctx->stream>>>(s->dP[s->cur], s->dmat, s->ncell); }));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    s->xstate = XS_NONE;
    return TDGL_OK;
}

int tdgl_set_material_map(tdgl_sim *s, const uint8_t *ids, int where) {
    if (!s || !ids || !valid_where(where)) return TDGL_EINVAL;
    ctx_set(s->ctx);
    if (where == TDGL_HOST) {
        memcpy(s->map.data(), ids, s->ncell);
    } else {
        CK(s->ctx, cudaMemcpy(s->map.data(), ids, s->ncell, cudaMemcpyDeviceToHost));
    }
    for (long i = 0; i < s->ncell; ++i)
        if (s->map[i] >= TDGL_MAX_MATERIALS) return fail(s->ctx, TDGL_EINVAL, "material id %d >= %d", (int)s->map[i], TDGL_MAX_MATERIALS);
    return apply_map(s);
}

int tdgl_set_layers(tdgl_sim *s, int n, const int *z0, const int *z1, const int *id) {
    if (!s || n < 0 || (n > 0 && (!z0 || !z1 || !id))) return TDGL_EINVAL;
    std::fill(s->map.begin(), s->map.end(), 0);
    const long plane = (long)s->nx * s->ny;
    for (int i = 0; i < n; ++i) {
        if (id[i] < 0 || id[i] >= TDGL_MAX_MATERIALS) return fail(s->ctx, TDGL_EINVAL, "layer id %d", id[i]);
        const int a = std::max(0, z0[i]), b = std::min(s->nz, z1[i]);
        for (int z = a; z < b; ++z) std::fill(s->map.begin() + z * plane, s->map.begin() + (z + 1) * plane, (uint8_t)id[i]);
    }
    return apply_map(s);
}

int tdgl_set_eps_b(tdgl_sim *s, double eps_b) {
    if (!s || !(eps_b > 0) || !std::isfinite(eps_b)) return s ? fail(s->ctx, TDGL_EINVAL, "eps_b must be > 0") : TDGL_EINVAL;
    if (eps_b != s->eps_b) s->xstate = (s->xstate == XS_EHAT) ? XS_NONE : s->xstate;
    s->eps_b = eps_b;
    s->ab_hist = 0;
    return TDGL_OK;
}

int tdgl_set_terms(tdgl_sim *s, unsigned mask) {
    if (!s || (mask & ~TDGL_TERM_ALL)) return TDGL_EINVAL;
    s->terms = mask;
    s->ab_hist = 0;
    return TDGL_OK;
}

int tdgl_set_temperature(tdgl_sim *s, double T) {
    if (!s || !(T > 0) || !std::isfinite(T)) return s ? fail(s->ctx, TDGL_EINVAL, "T must be > 0") : TDGL_EINVAL;
    s->T = T;
    s->dirty = true;
    return TDGL_OK;
}

int tdgl_set_field(tdgl_sim *s, double Ex, double Ey, double Ez) {
    if (!s || !std::isfinite(Ex) || !std::isfinite(Ey) || !std::isfinite(Ez)) return TDGL_EINVAL;
    s->E[0] = Ex; s->E[1] = Ey; s->E[2] = Ez;
    s->ab_hist = 0;
    return TDGL_OK;
}

int tdgl_set_field_ac(tdgl_sim *s, double Ax, double Ay, double Az, double freq_hz, double phase) {
    if (!s || !std::isfinite(Ax) || !std::isfinite(Ay) || !std::isfinite(Az) || !std::isfinite(freq_hz) ||
        !std::isfinite(phase) || freq_hz < 0)
        return s ? fail(s->ctx, TDGL_EINVAL, "bad AC field") : TDGL_EINVAL;
    s->Eac[0] = Ax; s->Eac[1] = Ay; s->Eac[2] = Az;
    s->ac_freq = freq_hz;
    s->ac_phase = phase;
    s->ab_hist = 0;
    return TDGL_OK;
}

int tdgl_set_integrator(tdgl_sim *s, int method) {
    if (!s || method < TDGL_EULER || method > TDGL_AB3M2)
        return s ? fail(s->ctx, TDGL_EINVAL, "integrator %d", method) : TDGL_EINVAL;
    ctx_set(s->ctx);
    if (method == TDGL_HEUN && !s->dhbuf) CK(s->ctx, cudaMalloc(&s->dhbuf, 3ull * s->ncell * sizeof(float)));
    if (method >= TDGL_RK45 && !s->dstage) {
        CK(s->ctx, cudaMalloc(&s->dstage, 6ull * 3 * s->ncell * sizeof(float)));
        CK(s->ctx, cudaMalloc(&s->derrmax, sizeof(unsigned)));
    }
    if (s->batch && method >= TDGL_RK45)
        return fail(s->ctx, TDGL_EINVAL, "RK45 and AB3M2 are not available for a sim inside a batch");
    s->integrator = method;
    s->ab_hist = 0;
    return TDGL_OK;
}

int tdgl_zpass_variant(tdgl_ctx *ctx, int length, int *variant, double *us) {
    const int vi = zvar_index(length);
    if (!ctx || !variant || vi < 0) return ctx ? fail(ctx, TDGL_EINVAL, "z-pass variants exist for 128, 256 and 512") : TDGL_EINVAL;
    *variant = ctx->zvar[vi];
    if (us)
        for (int v = 0; v < kZVariants; ++v) us[v] = ctx->zus[vi][v];
    return TDGL_OK;
}

int tdgl_set_zpass_variant(tdgl_ctx *ctx, int length, int variant) {
    const int vi = zvar_index(length);
    if (!ctx || vi < 0 || variant < -1 || variant >= zvar_count(length))
        return ctx ? fail(ctx, TDGL_EINVAL, "z-pass variant %d for length %d", variant, length) : TDGL_EINVAL;
    ctx->zvar[vi] = variant;
    if (variant < 0)
        for (int v = 0; v < kZVariants; ++v) ctx->zus[vi][v] = 0.0;
    return TDGL_OK;
}

int tdgl_row_tile(tdgl_sim *s, int *rows, int *candidates, double *us) {
    if (!s || !rows) return TDGL_EINVAL;
    *rows = s->row_tile;
    for (int i = 0; i < TDGL_ROW_CANDIDATES; ++i) {
        if (candidates) candidates[i] = s->row_cand[i];
        if (us) us[i] = s->row_us[i];
    }
    return TDGL_OK;
}

int tdgl_fft_pad(tdgl_sim *s, int *Mx, int *My, int *Mz) {
    if (!s || !Mx || !My || !Mz) return TDGL_EINVAL;
    *Mx = s->Mx;
    *My = s->My;
    *Mz = s->Mz;
    return TDGL_OK;
}

int tdgl_set_fft_pad(tdgl_sim *s, int Mx, int My, int Mz) {
    if (!s) return TDGL_EINVAL;
    tdgl_ctx *ctx = s->ctx;
    if (Mx == 0) Mx = default_x_length(s->nx);
    if (My == 0) My = default_y_length(s->ny);
    if (Mz == 0) Mz = default_z_length(s->nz);
    if (Mx < 2 * s->nx - 1 || My < 2 * s->ny - 1 || Mz < 2 * s->nz - 1 || Mx % 2 != 0 || !is_smooth(Mx) ||
        !is_smooth(My) || !is_smooth(Mz) || Mx > 4 * TDGL_MAX_DIM || My > 4 * TDGL_MAX_DIM || Mz > 4 * TDGL_MAX_DIM)
        return fail(ctx, TDGL_EINVAL, "padded lengths %d %d %d: each must be 2^a 3^b, at least 2n - 1 and at most %d "
                                      "(x even)", Mx, My, Mz, 4 * TDGL_MAX_DIM);
    if (Mx == s->Mx && My == s->My && Mz == s->Mz) return TDGL_OK;
    ctx_set(ctx);
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    for (auto &g : s->graphs) cudaGraphExecDestroy(g.exec);
    for (auto &g : s->relax_graphs) cudaGraphExecDestroy(g.exec);
    s->graphs.clear();
    s->relax_graphs.clear();
    if (s->batch) drop_cache(s->batch);   // its work lists hold this sim's items
    // spectra and the tensor spectrum are sized by the padded lengths: rebuilt on the next use
    cudaFree(s->dX); cudaFree(s->dY); cudaFree(s->dNhat);
    s->dX = s->dY = nullptr;
    s->dNhat = nullptr;
    s->spectra_alloc = false;
    s->tensor_ready = false;
    s->has_ymap = s->has_nmap = false;
    s->xstate = XS_NONE;
    s->ab_hist = 0;
    s->rows_tuned = false;
    s->row_tile = 0;
    std::vector<float2> tw;
    set_lengths(s, Mx, My, Mz, tw);
    cudaFree(s->dtw);
    s->dtw = nullptr;
    CK(ctx, cudaMalloc(&s->dtw, tw.size() * sizeof(float2)));
    CK(ctx, cudaMemcpy(s->dtw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice));
    return upload_items(s);
}

int tdgl_set_row_tile(tdgl_sim *s, int rows) {
    if (!s || rows < 0) return s ? fail(s->ctx, TDGL_EINVAL, "row tile %d", rows) : TDGL_EINVAL;
    tdgl_ctx *ctx = s->ctx;
    ctx_set(ctx);
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    // the captured step sequences hold the old row items: drop them (recaptured on the next use)
    for (auto &g : s->graphs) cudaGraphExecDestroy(g.exec);
    for (auto &g : s->relax_graphs) cudaGraphExecDestroy(g.exec);
    s->graphs.clear();
    s->relax_graphs.clear();
    s->row_tile = rows;
    s->rows_tuned = rows > 0;   // 0: tuned (or taken from the context's record) at the next preparation
    if (rows > 0)
        for (int i = 0; i < TDGL_ROW_CANDIDATES; ++i) {
            s->row_cand[i] = 0;
            s->row_us[i] = 0.0;
        }
    build_items(s);
    if (rows > 0) s->row_tile = std::min(rows, s->rows_cnt_max);
    return upload_items(s);
}

int tdgl_set_adaptive(tdgl_sim *s, double err_tol, double dt_min, double dt_max) {
    if (!s || !(err_tol >= 0) || !(dt_min >= 0) || !(dt_max >= 0) || !std::isfinite(err_tol) || !std::isfinite(dt_min) ||
        !std::isfinite(dt_max) || (dt_max > 0 && dt_max < dt_min))
        return s ? fail(s->ctx, TDGL_EINVAL, "bad adaptive step parameters") : TDGL_EINVAL;
    s->ad_tol = err_tol;
    s->ad_min = dt_min;
    s->ad_max = dt_max;
    s->dt_next = 0.0;
    return TDGL_OK;
}

int tdgl_get_dt(tdgl_sim *s, double *dt) {
    if (!s || !dt) return TDGL_EINVAL;
    *dt = s->dt_next;
    return TDGL_OK;
}

int tdgl_set_time(tdgl_sim *s, double t) {
    if (!s || !std::isfinite(t)) return TDGL_EINVAL;
    s->time = t;
    s->ab_hist = 0;
    return TDGL_OK;
}

int tdgl_get_time(tdgl_sim *s, double *t) {
    if (!s || !t) return TDGL_EINVAL;
    *t = s->time;
    return TDGL_OK;
}

int tdgl_set_scales(tdgl_sim *s, double P0, double alpha_ref) {
    if (!s || !(P0 > 0) || !(alpha_ref > 0) || !std::isfinite(P0) || !std::isfinite(alpha_ref)) return TDGL_EINVAL;
    ctx_set(s->ctx);
    const double old = s->scales_fixed ? s->P0 : 0.0;
    s->P0 = P0;
    s->alpha_ref = alpha_ref;
    s->dirty = true;
    if (old > 0 && old != P0) {
        const float f = (float)(old / P0);
        TRY(launch(s->ctx, TDGL_K_OTHER, [&] {
            k_scale_out<<<grid_for(3 * s->ncell), 256, 0, s->ctx->stream>>>(s->dP[s->cur], s->dP[s->cur], 3 * s->ncell, f);
        }));
        s->xstate = XS_NONE;
    }
    s->scales_fixed = true;
    return TDGL_OK;
}

int tdgl_get_scales(tdgl_sim *s, double *P0, double *alpha_ref) {
    if (!s) return TDGL_EINVAL;
    if (!s->scales_fixed && lowest_material(s)) fix_scales(s);
    if (P0) *P0 = s->P0;
    if (alpha_ref) *alpha_ref = s->alpha_ref;
    return TDGL_OK;
}

int tdgl_set_P(tdgl_sim *s, const float *P, int where) {
    if (!s || !P || !valid_where(where)) return TDGL_EINVAL;
    tdgl_ctx *ctx = s->ctx;
    ctx_set(ctx);
    if (lowest_material(s)) fix_scales(s);
    TRY(ensure_out(s));
    TRY(copy_in(ctx, s->dout, P, 3ull * s->ncell * sizeof(float), where));
    const float f = (float)(1.0 / s->P0);
    TRY(launch(ctx, TDGL_K_OTHER, [&] {
        k_scale_in<<<grid_for(3 * s->ncell), 256, 0, ctx->stream>>>(s->dP[s->cur], s->dout, s->dmat, s->ncell, f);
    }));
    if (where == TDGL_HOST) CK(ctx, cudaStreamSynchronize(ctx->stream));
    s->ab_hist = 0;
    s->xstate = XS_NONE;
    return TDGL_OK;
}

int tdgl_get_P(tdgl_sim *s, float *out, int where) {
    if (!s || !out || !valid_where(where)) return TDGL_EINVAL;
    tdgl_ctx *ctx = s->ctx;
    ctx_set(ctx);
    if (lowest_material(s)) fix_scales(s);
    TRY(ensure_out(s));
    const float f = (float)s->P0;
    TRY(launch(ctx, TDGL_K_OTHER, [&] {
        k_scale_out<<<grid_for(3 * s->ncell), 256, 0, ctx->stream>>>(s->dout, s->dP[s->cur], 3 * s->ncell, f);
    }));
    return copy_out(ctx, out, s->dout, 3ull * s->ncell * sizeof(float), where);
}

// ---- asynchronous host I/O -------------------------------------------------------------------
// Uploads run on the context's `up` stream into din_a, downloads on its `down` stream from dout_a;
// the scale kernels and the steps run on the context's stream.  Events order each staging buffer's
// writer after its previous reader, so consecutive upload / step / download calls overlap: the
// upload of the next input and the download of the previous result run during the current steps.
// Each direction alternates between two staging buffers, so an upload need not wait for the scale
// kernel of the one before it (nor a scale kernel for the download before it): the copies of one
// direction follow each other back to back.
int io_setup(tdgl_sim *s) {
    tdgl_ctx *ctx = s->ctx;
    if (!ctx->up) CK(ctx, cudaStreamCreateWithFlags(&ctx->up, cudaStreamNonBlocking));
    if (!ctx->down) CK(ctx, cudaStreamCreateWithFlags(&ctx->down, cudaStreamNonBlocking));
    for (int i = 0; i < 2; ++i)
        for (cudaEvent_t *e : {&s->ev_in_ready[i], &s->ev_in_free[i], &s->ev_out_ready[i], &s->ev_out_free[i]})
            if (!*e) CK(ctx, cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    return TDGL_OK;
}

int tdgl_set_P_async(tdgl_sim *s, const float *P) {
    if (!s || !P) return TDGL_EINVAL;
    tdgl_ctx *ctx = s->ctx;
    ctx_set(ctx);
    if (lowest_material(s)) fix_scales(s);
    TRY(io_setup(s));
    const size_t bytes = 3ull * s->ncell * sizeof(float);
    const int i = s->in_next;
    if (!s->din_a[i]) CK(ctx, cudaMalloc(&s->din_a[i], bytes));
    s->in_next ^= 1;
    // din_a[i] is free once the scale kernel of the upload before last (the one that used it) has
    // read it (an event never recorded counts as complete)
    CK(ctx, cudaStreamWaitEvent(ctx->up, s->ev_in_free[i], 0));
    CK(ctx, cudaMemcpyAsync(s->din_a[i], P, bytes, cudaMemcpyHostToDevice, ctx->up));
    CK(ctx, cudaEventRecord(s->ev_in_ready[i], ctx->up));
    CK(ctx, cudaStreamWaitEvent(ctx->stream, s->ev_in_ready[i], 0));
    const float f = (float)(1.0 / s->P0);
    TRY(launch(ctx, TDGL_K_OTHER, [&] {
        k_scale_in<<<grid_for(3 * s->ncell), 256, 0, ctx->stream>>>(s->dP[s->cur], s->din_a[i], s->dmat, s->ncell, f);
    }));
    CK(ctx, cudaEventRecord(s->ev_in_free[i], ctx->stream));
    s->ab_hist = 0;
    s->xstate = XS_NONE;
    return TDGL_OK;
}

int tdgl_get_P_async(tdgl_sim *s, float *out) {
    if (!s || !out) return TDGL_EINVAL;
    tdgl_ctx *ctx = s->ctx;
    ctx_set(ctx);
    if (lowest_material(s)) fix_scales(s);
    TRY(io_setup(s));
    const size_t bytes = 3ull * s->ncell * sizeof(float);
    const int i = s->out_next;
    if (!s->dout_a[i]) CK(ctx, cudaMalloc(&s->dout_a[i], bytes));
    s->out_next ^= 1;
    // dout_a[i] is free once the download before last (the one that used it) has read it
    CK(ctx, cudaStreamWaitEvent(ctx->stream, s->ev_out_free[i], 0));
    const float f = (float)s->P0;
    TRY(launch(ctx, TDGL_K_OTHER, [&] {
        k_scale_out<<<grid_for(3 * s->ncell), 256, 0, ctx->stream>>>(s->dout_a[i], s->dP[s->cur], 3 * s->ncell, f);
    }));
    CK(ctx, cudaEventRecord(s->ev_out_ready[i], ctx->stream));
    CK(ctx, cudaStreamWaitEvent(ctx->down, s->ev_out_ready[i], 0));
    CK(ctx, cudaMemcpyAsync(out, s->dout_a[i], bytes, cudaMemcpyDeviceToHost, ctx->down));
    CK(ctx, cudaEventRecord(s->ev_out_free[i], ctx->down));
    return TDGL_OK;
}

int tdgl_step_async(tdgl_sim *s, int n, double dt) {
    if (!s || n < 0 || !(dt > 0) || !std::isfinite(dt)) return s ? fail(s->ctx, TDGL_EINVAL, "bad n or dt") : TDGL_EINVAL;
    ctx_set(s->ctx);
    if (s->integrator >= TDGL_RK45)
        return fail(s->ctx, TDGL_EINVAL, "RK45 and AB3M2 read their error estimates on the host: use tdgl_step");
    if (n == 0) return TDGL_OK;
    TRY(prepare(s, s->terms));
    TRY(steps_nosync(s, n, dt));
    s->status_pending = true;
    return TDGL_OK;
}

int tdgl_sync(tdgl_sim *s) {
    if (!s) return TDGL_EINVAL;
    tdgl_ctx *ctx = s->ctx;
    ctx_set(ctx);
    // the context's stream holds every upload's scale kernel (after its copy) and every step;
    // the last download's event covers the downloads
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    for (int i = 0; i < 2; ++i)
        if (s->ev_out_free[i]) CK(ctx, cudaEventSynchronize(s->ev_out_free[i]));
    if (!s->status_pending) return TDGL_OK;
    s->status_pending = false;
    double m;
    int f;
    TRY(read_status(s, &m, &f));
    if (f) {
        CK(ctx, cudaMemsetAsync(s->dflag, 0, sizeof(int), ctx->stream));
        if (f & 2) return fail(ctx, TDGL_ETIMEOUT, "a bounded wait for a tensor copy timed out");
        return fail(ctx, TDGL_EDIVERGED, "P diverged (NaN or |P| > 1e3 P0)");
    }
    return TDGL_OK;
}

int tdgl_init_random(tdgl_sim *s, uint64_t seed, double amp) {
    if (!s || !(amp >= 0) || !std::isfinite(amp)) return TDGL_EINVAL;
    tdgl_ctx *ctx = s->ctx;
    ctx_set(ctx);
    if (lowest_material(s)) fix_scales(s);
    const float a = (float)(amp / s->P0);
    TRY(launch(ctx, TDGL_K_OTHER, [&] {
        k_init_random<<<grid_for(3 * s->ncell), 256, 0, ctx->stream>>>(s->dP[s->cur], s->dmat, s->ncell,
                                                                         (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32), a);
    }));
    s->ab_hist = 0;
    s->xstate = XS_NONE;
    return TDGL_OK;
}

int tdgl_get_field(tdgl_sim *s, unsigned mask, float *out, int where) {
    if (!s || !out || !valid_where(where) || (mask & ~TDGL_TERM_ALL)) return TDGL_EINVAL;
    tdgl_ctx *ctx = s->ctx;
    ctx_set(ctx);
    TRY(prepare(s, mask));
    TRY(ensure_out(s));
    fill_desc(s, 0.0, mask);
    TRY(upload_desc(s));
    const bool elec = (mask & TDGL_TERM_ELEC) != 0;
    Work w = sim_work(s, elec);
    if (elec) TRY(ensure_ehat(s, w));
    TRY(launch_rows(ctx, MODE_FIELD, w, 0));
    return copy_out(ctx, out, s->dout, 3ull * s->ncell * sizeof(float), where);
}

int tdgl_step(tdgl_sim *s, int n, double dt) {
    if (!s || n < 0 || !(dt > 0) || !std::isfinite(dt)) return s ? fail(s->ctx, TDGL_EINVAL, "bad n or dt") : TDGL_EINVAL;
    ctx_set(s->ctx);
    if (n == 0) return TDGL_OK;
    const bool changed = s->dirty;
    TRY(prepare(s, s->terms));
    if (s->integrator >= TDGL_RK45) {
        if (changed) s->ab_hist = 0;
        double m;
        return multistage_steps(s, n, dt, &m);
    }
    TRY(steps_nosync(s, n, dt));
    double m;
    int f;
    TRY(read_status(s, &m, &f));
    if (f) {
        CK(s->ctx, cudaMemsetAsync(s->dflag, 0, sizeof(int), s->ctx->stream));
        if (f & 2) return fail(s->ctx, TDGL_ETIMEOUT, "a bounded wait for a tensor copy timed out");
        return fail(s->ctx, TDGL_EDIVERGED, "P diverged (NaN or |P| > 1e3 P0)");
    }
    return TDGL_OK;
}

int tdgl_last_max_dP(tdgl_sim *s, double *out) {
    if (!s || !out) return TDGL_EINVAL;
    *out = s->last_maxdp;
    return TDGL_OK;
}

// Relaxation with its convergence loop on the device: one CUDA graph whose conditional WHILE
// node repeats a body of k steps (the launches of steps_nosync) followed by k_relax_check, which
// counts the steps and clears the loop condition once max|dP*| of the body's last step is below
// tol, a kernel raised the divergence or timeout flag, or another body would pass max_steps.  The
// host waits once per call instead of once per k steps; the steps taken and the final state are
// those of the host-checked loop.  Usable for Euler with even k (P returns to the same buffer
// after each body, so one descriptor serves every iteration) and for Heun, without a
// time-dependent applied field (the body replays the same launch indices).
// End of one loop body: count its k steps and keep looping while no kernel raised a flag, the
// last step's max |dP*| (float bits in maxdp) is not below tol and another body fits under the cap.
__global__ void k_relax_check(cudaGraphConditionalHandle h, RelaxState *st, const unsigned *maxdp, const int *flag) {
    const long done = st->done + st->k;
    st->done = done;
    const unsigned u = *maxdp;
    const bool conv = u < 0x7f800000u && (double)__uint_as_float(u) < st->tol;
    const bool more = *flag == 0 && !conv && done + st->k <= st->max_steps;
    cudaGraphSetConditional(h, more ? 1u : 0u);
}

bool relax_on_device_ok(const tdgl_sim *s, int k) {
    const bool ac = s->ac_freq != 0.0 && (s->Eac[0] != 0.0 || s->Eac[1] != 0.0 || s->Eac[2] != 0.0);
    const bool parity_ok = s->integrator == TDGL_HEUN || (s->integrator == TDGL_EULER && (k & 1) == 0);
    return parity_ok && !ac && !s->ctx->profiling && s->ctx->stream != nullptr;
}

int relax_on_device(tdgl_sim *s, double dt, double tol, long max_steps, int k, long *done, double *maxdp, int *flag) {
    tdgl_ctx *ctx = s->ctx;
    const bool elec = (s->terms & TDGL_TERM_ELEC) != 0;
    const bool heun = s->integrator == TDGL_HEUN;
    fill_desc(s, dt, s->terms);
    TRY(upload_desc(s));
    Work w = sim_work(s, elec);
    if (elec && s->xstate != XS_PHAT) {   // the body starts from P-hat of the current P
        TRY(launch_rows(ctx, MODE_XFWD, w, 0));
        s->xstate = XS_PHAT;
    }
    if (!s->drelax) CK(ctx, cudaMalloc(&s->drelax, sizeof(RelaxState)));
    tdgl_sim::GraphRec *G = nullptr;
    for (auto &g : s->relax_graphs)
        if (g.n == k && g.elec == elec && g.integ == s->integrator) G = &g;
    if (!G) {
        cudaGraph_t g = nullptr;
        CK(ctx, cudaGraphCreate(&g, 0));
        cudaGraphConditionalHandle h;
        cudaGraphNodeParams np = {};
        cudaGraphNode_t node;
        cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 1u, cudaGraphCondAssignDefault);
        if (e == cudaSuccess) {
            np.type = cudaGraphNodeTypeConditional;
            np.conditional.handle = h;
            np.conditional.type = cudaGraphCondTypeWhile;
            np.conditional.size = 1;
            e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
        }
        if (e != cudaSuccess) {
            cudaGraphDestroy(g);
            CK(ctx, e);
        }
        cudaGraph_t body = np.conditional.phGraph_out[0];
        const long l0 = ctx->launches;
        CK(ctx, cudaStreamBeginCaptureToGraph(ctx->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        int rc = record_steps(s, w, 0, k, elec, heun);
        if (rc == TDGL_OK)
            rc = launch(ctx, TDGL_K_OTHER, [&] { k_relax_check<<<1, 1, 0, ctx->stream>>>(h, s->drelax, s->dmaxdp, s->dflag); });
        cudaGraph_t captured = nullptr;
        e = cudaStreamEndCapture(ctx->stream, &captured);
        const long kernels = ctx->launches - l0;
        ctx->launches = l0;
        cudaGraphExec_t exec = nullptr;
        if (rc == TDGL_OK && e == cudaSuccess) e = cudaGraphInstantiate(&exec, g, 0);
        cudaGraphDestroy(g);
        if (rc != TDGL_OK) return rc;
        CK(ctx, e);
        s->relax_graphs.push_back(tdgl_sim::GraphRec{k, elec, 0, s->integrator, exec, kernels});
        G = &s->relax_graphs.back();
    }
    RelaxState st{0, max_steps, tol, k};
    CK(ctx, cudaMemcpyAsync(s->drelax, &st, sizeof st, cudaMemcpyHostToDevice, ctx->stream));
    CK(ctx, cudaGraphLaunch(G->exec, ctx->stream));
    CK(ctx, cudaMemcpyAsync(&st, s->drelax, sizeof st, cudaMemcpyDeviceToHost, ctx->stream));
    TRY(read_status(s, maxdp, flag));     // synchronizes
    *done = st.done;
    ctx->launches += (st.done / k) * G->kernels;
    for (long c = 0; c < st.done / k; ++c) s->time += k * dt;   // as the host loop adds it
    s->xstate = elec ? XS_PHAT : XS_NONE;
    return TDGL_OK;
}

int tdgl_relax(tdgl_sim *s, double dt, double tol, long max_steps, int check_every, long *steps_taken) {
    if (steps_taken) *steps_taken = 0;
    if (!s || !(dt > 0) || !(tol > 0) || max_steps < 0 || check_every < 1) return TDGL_EINVAL;
    ctx_set(s->ctx);
    const bool changed = s->dirty;
    TRY(prepare(s, s->terms));
    long done = 0;
    if (s->integrator >= TDGL_RK45) {
        if (changed) s->ab_hist = 0;
        while (done < max_steps) {
            const long k = std::min<long>(check_every, max_steps - done);
            double m;
            TRY(multistage_steps(s, k, dt, &m));
            done += k;
            if (steps_taken) *steps_taken = done;
            if (m < tol) return TDGL_OK;
        }
        return fail(s->ctx, TDGL_ENOTCONVERGED, "not converged after %ld steps (last max|dP| = %g P0)", done,
                    s->last_maxdp);
    }
    auto flagged = [&](int f) {
        CK(s->ctx, cudaMemsetAsync(s->dflag, 0, sizeof(int), s->ctx->stream));
        if (f & 2) return fail(s->ctx, TDGL_ETIMEOUT, "a bounded wait for a tensor copy timed out");
        return fail(s->ctx, TDGL_EDIVERGED, "P diverged after %ld steps", done);
    };
    const bool elec = (s->terms & TDGL_TERM_ELEC) != 0;
    while (done < max_steps) {
        // whole chunks on the device, unless the field spectrum of the current P is already in X
        // (left by an energy or field call): the host-checked chunk's first step uses it
        if (max_steps - done >= check_every && relax_on_device_ok(s, check_every) && !(elec && s->xstate == XS_EHAT)) {
            long d = 0;
            double m;
            int f;
            TRY(relax_on_device(s, dt, tol, max_steps - done, check_every, &d, &m, &f));
            done += d;
            if (steps_taken) *steps_taken = done;
            if (f) return flagged(f);
            if (m < tol) return TDGL_OK;
            continue;   // fewer than check_every steps remain
        }
        const int k = (int)std::min<long>(check_every, max_steps - done);
        TRY(steps_nosync(s, k, dt));
        done += k;
        double m;
        int f;
        TRY(read_status(s, &m, &f));
        if (steps_taken) *steps_taken = done;
        if (f) return flagged(f);
        if (m < tol) return TDGL_OK;
    }
    return fail(s->ctx, TDGL_ENOTCONVERGED, "not converged after %ld steps (last max|dP| = %g P0)", done, s->last_maxdp);
}

int tdgl_energy(tdgl_sim *s, tdgl_energies *out) {
    if (!s || !out) return TDGL_EINVAL;
    tdgl_ctx *ctx = s->ctx;
    ctx_set(ctx);
    TRY(prepare(s, s->terms));
    fill_desc(s, 0.0, s->terms);
    TRY(upload_desc(s));
    const bool elec = (s->terms & TDGL_TERM_ELEC) != 0;
    Work w = sim_work(s, elec);
    if (elec) TRY(ensure_ehat(s, w));
    CK(ctx, cudaMemsetAsync(s->denergy, 0, 4 * sizeof(double), ctx->stream));
    TRY(launch_rows(ctx, MODE_ENERGY, w, 0));
    double e[4];
    CK(ctx, cudaMemcpyAsync(e, s->denergy, sizeof e, cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    const double scale = s->alpha_ref * s->P0 * s->P0 * s->d[0] * s->d[1] * s->d[2];
    out->land = e[0] * scale;
    out->grad = e[1] * scale;
    out->elec = e[2] * scale;
    out->ext = e[3] * scale;
    out->total = out->land + out->grad + out->elec + out->ext;
    return TDGL_OK;
}

// ---- batches ---------------------------------------------------------------------------------------
int tdgl_batch_create(tdgl_ctx *ctx, int n, tdgl_sim *const *sims, tdgl_batch **out) {
    if (!ctx || !out || n < 1 || !sims) return TDGL_EINVAL;
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        if (!sims[i] || sims[i]->ctx != ctx) return fail(ctx, TDGL_EINVAL, "sim %d missing or of another context", i);
        if (sims[i]->batch) return fail(ctx, TDGL_ESTATE, "sim %d already in a batch", i);
        for (int j = 0; j < i; ++j)
            if (sims[j] == sims[i]) return fail(ctx, TDGL_EINVAL, "sim %d listed twice", i);
    }
    ctx_set(ctx);
    tdgl_batch *b = new tdgl_batch();
    b->ctx = ctx;
    b->sims.assign(sims, sims + n);
    if (cudaMalloc(&b->ddescs, n * sizeof(SimDev)) != cudaSuccess) {
        delete b;
        return fail(ctx, TDGL_ENOMEM, "batch descriptors");
    }
    for (auto s : b->sims) s->batch = b;
    ctx->batches.push_back(b);
    *out = b;
    return TDGL_OK;
}

// work lists and captured step sequences of a batch for one active set
struct tdgl_batch::Cached {
    Work w;
    struct G {
        int n;
        bool heun;
        cudaGraphExec_t exec;
        long kernels;
    };
    std::vector<G> graphs;
    // the device relaxation loop over this active set (k steps per body, integrator)
    cudaGraphExec_t relax_exec = nullptr;
    int relax_k = 0;
    bool relax_heun = false;
    long relax_kernels = 0;
    ~Cached() {
        for (auto &g : graphs) cudaGraphExecDestroy(g.exec);
        if (relax_exec) cudaGraphExecDestroy(relax_exec);
    }
};

extern "C++" {
static void drop_cache(tdgl_batch *b) {
    delete b->cache;
    b->cache = nullptr;
}
}

void tdgl_batch_destroy(tdgl_batch *b) {
    if (!b) return;
    ctx_set(b->ctx);
    cudaStreamSynchronize(b->ctx->stream);
    for (auto s : b->sims) s->batch = nullptr;
    auto &v = b->ctx->batches;
    v.erase(std::remove(v.begin(), v.end(), b), v.end());
    drop_cache(b);
    cudaFree(b->ddescs);
    cudaFree(b->d_items);
    cudaFree(b->drelax);
    cudaFree(b->dmember);
    cudaFree(b->dstatus);
    cudaFree(b->dsteps);
    delete b;
}


namespace {

using GroupList = std::vector<std::pair<int, std::vector<int4>>>;

size_t group_of(GroupList &g, std::vector<size_t> &sm, int N) {
    for (size_t i = 0; i < g.size(); ++i)
        if (g[i].first == N) return i;
    g.push_back({N, {}});
    sm.push_back(0);
    return g.size() - 1;
}

// concatenated work lists (row, y, z by transform length) of the active sims of a batch
int build_batch_work(tdgl_batch *b, const std::vector<int> &active, Work &w) {
    tdgl_ctx *ctx = b->ctx;
    GroupList rgr, ygr, zgr;
    std::vector<size_t> rsm, ysm, zsm;
    for (int idx : active) {
        tdgl_sim *s = b->sims[idx];
        const bool elec = (s->terms & TDGL_TERM_ELEC) != 0;
        const size_t gr = group_of(rgr, rsm, row_group_len(s));
        for (auto it : s->it_rows_full) rgr[gr].second.push_back(make_int4(idx, it.y, it.z, it.w));
        rsm[gr] = std::max(rsm[gr], smem_rows(s, s->rows_cnt_max));
        if (elec) {
            const size_t gy = group_of(ygr, ysm, s->yN), gz = group_of(zgr, zsm, s->zN);
            for (auto it : s->it_y) ygr[gy].second.push_back(make_int4(idx, it.y, it.z, it.w));
            for (auto it : s->it_z) zgr[gz].second.push_back(make_int4(idx, it.y, it.z, it.w));
            if (!s->yN) ysm[gy] = std::max(ysm[gy], smem_y(s, s->ky_cnt_max));
            if (!s->zN) zsm[gz] = std::max(zsm[gz], smem_z(s, s->kz_cnt_max));
        }
    }
    size_t tot = 0;
    for (auto &g : rgr) tot += g.second.size();
    for (auto &g : ygr) tot += g.second.size();
    for (auto &g : zgr) tot += g.second.size();
    if (tot > b->items_cap) {
        CK(ctx, cudaStreamSynchronize(ctx->stream));
        cudaFree(b->d_items);
        b->d_items = nullptr;
        CK(ctx, cudaMalloc(&b->d_items, tot * sizeof(int4)));
        b->items_cap = tot;
    }
    std::vector<int4> all;
    all.reserve(tot);
    w.descs = b->ddescs;
    auto emit = [&](GroupList &gl, std::vector<size_t> &sm, std::vector<Group> &out) {
        for (size_t i = 0; i < gl.size(); ++i) {
            out.push_back(Group{gl[i].first, b->d_items + all.size(), (int)gl[i].second.size(), sm[i]});
            all.insert(all.end(), gl[i].second.begin(), gl[i].second.end());
        }
    };
    emit(rgr, rsm, w.rg);
    emit(ygr, ysm, w.yg);
    emit(zgr, zsm, w.zg);
    CK(ctx, cudaMemcpyAsync(b->d_items, all.data(), tot * sizeof(int4), cudaMemcpyHostToDevice, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));   // the host vector goes out of scope
    return TDGL_OK;
}

// n steps of every active sim of a batch (one launch per kernel family and length class)
// Descriptors of the active sims (the others zeroed), work lists of the active set, the x-forward
// prologue of sims whose x-spectrum is not P-hat of their P, cleared flags: the state every
// step sequence of the batch starts from.
int batch_setup(tdgl_batch *b, const std::vector<int> &active, const double *dt) {
    tdgl_ctx *ctx = b->ctx;
    std::vector<SimDev> descs(b->sims.size());
    memset(descs.data(), 0, descs.size() * sizeof(SimDev));
    for (int idx : active) {
        fill_desc(b->sims[idx], dt[idx], b->sims[idx]->terms);
        descs[idx] = b->sims[idx]->desc;
    }
    CK(ctx, cudaMemcpyAsync(b->ddescs, descs.data(), descs.size() * sizeof(SimDev), cudaMemcpyHostToDevice, ctx->stream));
    if (!b->cache || b->w_active != active) {
        delete b->cache;
        b->cache = new tdgl_batch::Cached();
        b->w_active = active;
        TRY(build_batch_work(b, active, b->cache->w));
    }
    const Work &w = b->cache->w;
    // prologue: sims whose x-spectrum is not P-hat of the current P get the x forward pass
    {
        GroupList pgr;
        std::vector<size_t> psm;
        size_t npro = 0;
        for (int idx : active) {
            tdgl_sim *s = b->sims[idx];
            if ((s->terms & TDGL_TERM_ELEC) && s->xstate != XS_PHAT) {
                const size_t g = group_of(pgr, psm, row_group_len(s));
                for (auto it : s->it_rows_full) pgr[g].second.push_back(make_int4(idx, it.y, it.z, it.w));
                psm[g] = std::max(psm[g], smem_rows(s, s->rows_cnt_max));
                npro += s->it_rows_full.size();
            }
        }
        if (npro) {
            std::vector<int4> pro;
            pro.reserve(npro);
            int4 *dpro = nullptr;
            CK(ctx, cudaMalloc(&dpro, npro * sizeof(int4)));
            Work wp;
            wp.descs = w.descs;
            for (size_t i = 0; i < pgr.size(); ++i) {
                wp.rg.push_back(Group{pgr[i].first, dpro + pro.size(), (int)pgr[i].second.size(), psm[i]});
                pro.insert(pro.end(), pgr[i].second.begin(), pgr[i].second.end());
            }
            CK(ctx, cudaMemcpyAsync(dpro, pro.data(), npro * sizeof(int4), cudaMemcpyHostToDevice, ctx->stream));
            TRY(launch_rows(ctx, MODE_XFWD, wp, 0));
            CK(ctx, cudaStreamSynchronize(ctx->stream));
            cudaFree(dpro);
        }
    }
    for (int idx : active) CK(ctx, cudaMemsetAsync(b->sims[idx]->dflag, 0, sizeof(int), ctx->stream));
    return TDGL_OK;
}

// the launches of n steps of the active set (one per kernel family and length class)
int record_batch_steps(tdgl_batch *b, const std::vector<int> &active, int n) {
    tdgl_ctx *ctx = b->ctx;
    const Work &w = b->cache->w;
    const bool heun = b->sims[active[0]]->integrator == TDGL_HEUN;
    for (int i = 0; i < n; ++i) {
        TRY(launch_conv(ctx, w));
        if (heun) {
            TRY(launch_rows(ctx, MODE_HEUN1, w, 2 * i));
            TRY(launch_conv(ctx, w));
        }
        if (i == n - 1)
            for (int idx : active) CK(ctx, cudaMemsetAsync(b->sims[idx]->dmaxdp, 0, sizeof(unsigned), ctx->stream));
        TRY(launch_rows(ctx, heun ? MODE_HEUN2 : MODE_STEP, w, heun ? 2 * i + 2 : i));
    }
    return TDGL_OK;
}

// n steps of every active sim of a batch
int batch_steps(tdgl_batch *b, const std::vector<int> &active, int n, const double *dt) {
    tdgl_ctx *ctx = b->ctx;
    TRY(batch_setup(b, active, dt));
    const bool heun = b->sims[active[0]]->integrator == TDGL_HEUN;
    auto record = [&]() -> int { return record_batch_steps(b, active, n); };
    if (n >= 2 && !(n & 1) && !ctx->profiling && ctx->stream) {
        tdgl_batch::Cached::G *G = nullptr;
        for (auto &g : b->cache->graphs)
            if (g.n == n && g.heun == heun) G = &g;
        if (!G) {
            tdgl_batch::Cached::G r{n, heun, nullptr, 0};
            TRY(capture_graph(ctx, record, &r.exec, &r.kernels));
            b->cache->graphs.push_back(r);
            G = &b->cache->graphs.back();
        }
        CK(ctx, cudaGraphLaunch(G->exec, ctx->stream));
        ctx->launches += G->kernels;
    } else {
        TRY(record());
    }
    for (int idx : active) {
        tdgl_sim *s = b->sims[idx];
        if ((n & 1) && !heun) s->cur ^= 1;
        s->xstate = (s->terms & TDGL_TERM_ELEC) ? XS_PHAT : XS_NONE;
        s->time += n * dt[idx];
    }
    return TDGL_OK;
}

}  // namespace

static int batch_check_integrator(tdgl_batch *b) {
    for (auto s : b->sims) {
        if (s->integrator != b->sims[0]->integrator)
            return fail(b->ctx, TDGL_EINVAL, "sims of a batch must use one integrator");
        if (s->integrator >= TDGL_RK45) return fail(b->ctx, TDGL_EINVAL, "batches step with Euler or Heun");
    }
    return TDGL_OK;
}

int tdgl_batch_step(tdgl_batch *b, int n, const double *dt) {
    if (!b || n < 0 || !dt) return TDGL_EINVAL;
    tdgl_ctx *ctx = b->ctx;
    ctx_set(ctx);
    if (b->sims.empty()) return TDGL_OK;
    TRY(batch_check_integrator(b));
    std::vector<int> active;
    for (size_t i = 0; i < b->sims.size(); ++i) {
        if (!(dt[i] > 0) || !std::isfinite(dt[i])) return fail(ctx, TDGL_EINVAL, "dt[%zu]", i);
        TRY(prepare(b->sims[i], b->sims[i]->terms));
        active.push_back((int)i);
    }
    if (n == 0) return TDGL_OK;
    for (int done = 0; done < n;) {   // chunks as for a single sim (steps_nosync)
        const int len = std::min(kStepChunk, n - done);
        TRY(batch_steps(b, active, len, dt));
        done += len;
    }
    int rc = TDGL_OK;
    for (int idx : active) {
        double m;
        int f;
        TRY(read_status(b->sims[idx], &m, &f));
        if (f) rc = (f & 2) ? fail(ctx, TDGL_ETIMEOUT, "sim %d: a bounded wait timed out", idx)
                      : fail(ctx, TDGL_EDIVERGED, "sim %d diverged", idx);
    }
    return rc;
}

// Batch relaxation with its convergence loop on the device.  One CUDA graph per active set: a
// conditional WHILE node repeats a body of k steps of the whole active set followed by
// k_batch_check, which retires each running member whose last step's max |dP*| is below tol (or
// whose flag is raised) by setting skip in its descriptor: from the next body on, every kernel's
// blocks of that member return at once.  The loop hands back to the host when no member runs, when
// another body would pass the cap, or when the retired members hold a quarter of the active cells
// (the host then builds work lists without them).  Members stop at the same step as in the
// host-checked loop, so the results are identical.
__global__ void k_batch_check(cudaGraphConditionalHandle h, BatchRelaxState *st, SimDev *descs, const int *member,
                              long *steps, int *status) {
    __shared__ int s_running;
    __shared__ unsigned long long s_retired;
    const long done = st->done + st->k;
    if (threadIdx.x == 0) { s_running = 0; s_retired = 0ull; }
    __syncthreads();
    for (int i = threadIdx.x; i < st->n; i += blockDim.x) {
        if (!member[i] || descs[i].skip) continue;
        const unsigned u = *descs[i].maxdp;
        const int f = *descs[i].flag;
        const bool conv = u < 0x7f800000u && (double)__uint_as_float(u) < st->tol;
        if (f != 0 || conv) {
            descs[i].skip = 1;
            status[i] = (f & 2) ? 3 : (f != 0 ? 2 : 1);
            steps[i] = done;
            steps[st->n + i] = (long)u;     // the last step's max |dP*| (later bodies clear maxdp)
            atomicAdd(&s_retired, (unsigned long long)descs[i].ncell);
        } else {
            atomicAdd(&s_running, 1);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        st->done = done;
        st->cells_retired += (long)s_retired;
        const bool more = s_running > 0 && done + st->k <= st->max_steps && st->cells_retired < st->cells_stop;
        cudaGraphSetConditional(h, more ? 1u : 0u);
    }
}

bool batch_relax_on_device_ok(const tdgl_batch *b, const std::vector<int> &active, int k) {
    if (b->ctx->profiling || !b->ctx->stream) return false;
    for (int idx : active)
        if (!relax_on_device_ok(b->sims[idx], k)) return false;
    return true;
}

// One launch of the device loop over the active set, at most max_more steps.  On return: *done =
// steps the loop ran; for every member status[i], and for retired members steps[i] (steps run) and
// steps[n + i] (float bits of their last step's max |dP*|).
int batch_relax_on_device(tdgl_batch *b, const std::vector<int> &active, const double *dt, double tol, long max_more,
                          int k, long *done, std::vector<int> &status, std::vector<long> &steps) {
    tdgl_ctx *ctx = b->ctx;
    const int n = (int)b->sims.size();
    TRY(batch_setup(b, active, dt));
    const bool heun = b->sims[active[0]]->integrator == TDGL_HEUN;
    if (!b->drelax) {
        CK(ctx, cudaMalloc(&b->drelax, sizeof(BatchRelaxState)));
        CK(ctx, cudaMalloc(&b->dmember, n * sizeof(int)));
        CK(ctx, cudaMalloc(&b->dstatus, n * sizeof(int)));
        CK(ctx, cudaMalloc(&b->dsteps, 2ull * n * sizeof(long)));
    }
    tdgl_batch::Cached &C = *b->cache;
    if (!C.relax_exec || C.relax_k != k || C.relax_heun != heun) {
        if (C.relax_exec) cudaGraphExecDestroy(C.relax_exec);
        C.relax_exec = nullptr;
        cudaGraph_t g = nullptr;
        CK(ctx, cudaGraphCreate(&g, 0));
        cudaGraphConditionalHandle h;
        cudaGraphNodeParams np = {};
        cudaGraphNode_t node;
        cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 1u, cudaGraphCondAssignDefault);
        if (e == cudaSuccess) {
            np.type = cudaGraphNodeTypeConditional;
            np.conditional.handle = h;
            np.conditional.type = cudaGraphCondTypeWhile;
            np.conditional.size = 1;
            e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
        }
        if (e != cudaSuccess) {
            cudaGraphDestroy(g);
            CK(ctx, e);
        }
        cudaGraph_t body = np.conditional.phGraph_out[0];
        const long l0 = ctx->launches;
        CK(ctx, cudaStreamBeginCaptureToGraph(ctx->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        int rc = record_batch_steps(b, active, k);
        if (rc == TDGL_OK)
            rc = launch(ctx, TDGL_K_OTHER, [&] {
                k_batch_check<<<1, 256, 0, ctx->stream>>>(h, b->drelax, b->ddescs, b->dmember, b->dsteps, b->dstatus);
            });
        cudaGraph_t captured = nullptr;
        e = cudaStreamEndCapture(ctx->stream, &captured);
        C.relax_kernels = ctx->launches - l0;
        ctx->launches = l0;
        cudaGraphExec_t exec = nullptr;
        if (rc == TDGL_OK && e == cudaSuccess) e = cudaGraphInstantiate(&exec, g, 0);
        cudaGraphDestroy(g);
        if (rc != TDGL_OK) return rc;
        CK(ctx, e);
        C.relax_exec = exec;
        C.relax_k = k;
        C.relax_heun = heun;
    }
    std::vector<int> member(n, 0);
    long cells = 0;
    for (int idx : active) {
        member[idx] = 1;
        cells += b->sims[idx]->ncell;
    }
    status.assign(n, 0);
    steps.assign(2 * n, 0);
    BatchRelaxState st{0, max_more, tol, k, n, 0, std::max(1L, cells / 4)};
    CK(ctx, cudaMemcpyAsync(b->drelax, &st, sizeof st, cudaMemcpyHostToDevice, ctx->stream));
    CK(ctx, cudaMemcpyAsync(b->dmember, member.data(), n * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    CK(ctx, cudaMemsetAsync(b->dstatus, 0, n * sizeof(int), ctx->stream));
    CK(ctx, cudaMemsetAsync(b->dsteps, 0, 2ull * n * sizeof(long), ctx->stream));
    CK(ctx, cudaGraphLaunch(C.relax_exec, ctx->stream));
    CK(ctx, cudaMemcpyAsync(&st, b->drelax, sizeof st, cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaMemcpyAsync(status.data(), b->dstatus, n * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaMemcpyAsync(steps.data(), b->dsteps, 2ull * n * sizeof(long), cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    *done = st.done;
    ctx->launches += (st.done / k) * C.relax_kernels;
    std::vector<unsigned> us(n, 0u);
    for (int idx : active)
        CK(ctx, cudaMemcpyAsync(&us[idx], b->sims[idx]->dmaxdp, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    for (int idx : active) {
        tdgl_sim *s = b->sims[idx];
        const long ran = status[idx] ? steps[idx] : st.done;
        s->time += ran * dt[idx];
        s->xstate = (s->terms & TDGL_TERM_ELEC) ? XS_PHAT : XS_NONE;
        const unsigned u = status[idx] ? (unsigned)steps[n + idx] : us[idx];
        float v;
        memcpy(&v, &u, sizeof v);
        s->last_maxdp = (u >= 0x7f800000u) ? INFINITY : (double)v;
    }
    return TDGL_OK;
}

int tdgl_batch_relax(tdgl_batch *b, const double *dt, double tol, long max_steps, int check_every,
                     long *steps_taken) {
    return tdgl_batch_relax_state(b, dt, tol, max_steps, check_every, steps_taken, nullptr);
}

int tdgl_batch_relax_state(tdgl_batch *b, const double *dt, double tol, long max_steps, int check_every,
                           long *steps_taken, int *state) {
    if (!b || !dt || !(tol > 0) || max_steps < 0 || check_every < 1) return TDGL_EINVAL;
    tdgl_ctx *ctx = b->ctx;
    ctx_set(ctx);
    const int n = (int)b->sims.size();
    if (n == 0) return TDGL_OK;
    TRY(batch_check_integrator(b));
    std::vector<int> active;
    std::vector<long> taken(n, 0);
    std::vector<int> st(n, TDGL_RELAX_CONVERGED);
    for (int i = 0; i < n; ++i) {
        if (!(dt[i] > 0) || !std::isfinite(dt[i])) return fail(ctx, TDGL_EINVAL, "dt[%d]", i);
        TRY(prepare(b->sims[i], b->sims[i]->terms));
        active.push_back(i);
    }
    long done = 0;
    int rc = TDGL_OK;
    // the device loop while whole check intervals remain, then host-checked chunks
    if (batch_relax_on_device_ok(b, active, check_every)) {
        while (!active.empty() && max_steps - done >= check_every) {
            long ran = 0;
            std::vector<int> status;
            std::vector<long> steps;
            TRY(batch_relax_on_device(b, active, dt, tol, max_steps - done, check_every, &ran, status, steps));
            std::vector<int> keep;
            for (int idx : active) {
                if (status[idx] == 0) {
                    taken[idx] = done + ran;
                    keep.push_back(idx);
                    continue;
                }
                taken[idx] = done + steps[idx];
                if (status[idx] == 2) {
                    st[idx] = TDGL_RELAX_DIVERGED;
                    rc = fail(ctx, TDGL_EDIVERGED, "sim %d diverged", idx);
                }
                if (status[idx] == 3) {
                    st[idx] = TDGL_RELAX_TIMEOUT;
                    rc = fail(ctx, TDGL_ETIMEOUT, "sim %d: a bounded wait timed out", idx);
                }
            }
            done += ran;
            active.swap(keep);
        }
    }
    while (!active.empty() && done < max_steps) {
        const int k = (int)std::min<long>(check_every, max_steps - done);
        TRY(batch_steps(b, active, k, dt));
        done += k;
        std::vector<int> keep;
        for (int idx : active) {
            double m;
            int f;
            TRY(read_status(b->sims[idx], &m, &f));
            taken[idx] = done;
            if (f) {
                st[idx] = (f & 2) ? TDGL_RELAX_TIMEOUT : TDGL_RELAX_DIVERGED;
                rc = (f & 2) ? fail(ctx, TDGL_ETIMEOUT, "sim %d: a bounded wait timed out", idx)
                             : fail(ctx, TDGL_EDIVERGED, "sim %d diverged", idx);
                continue;
            }
            if (!(m < tol)) keep.push_back(idx);
        }
        active.swap(keep);
    }
    for (int idx : active) st[idx] = TDGL_RELAX_AT_CAP;
    if (steps_taken)
        for (int i = 0; i < n; ++i) steps_taken[i] = taken[i];
    if (state)
        for (int i = 0; i < n; ++i) state[i] = st[i];
    if (rc != TDGL_OK) return rc;
    if (!active.empty()) return fail(ctx, TDGL_ENOTCONVERGED, "%zu sims not converged after %ld steps", active.size(), done);
    return TDGL_OK;
}

// ---- measurement -------------------------------------------------------------------------------------
int tdgl_profile(tdgl_ctx *ctx, int enable) {
    if (!ctx) return TDGL_EINVAL;
    ctx->profiling = enable != 0;
    return TDGL_OK;
}

int tdgl_profile_read(tdgl_ctx *ctx, int kind, double *total_ms, long *launches) {
    if (!ctx || kind < 0 || kind >= TDGL_K_COUNT) return TDGL_EINVAL;
    ctx_set(ctx);
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    for (auto &r : ctx->recs) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.a, r.b);
        ctx->prof_ms[r.kind] += ms;
        ctx->prof_n[r.kind] += 1;
        ctx->pool.push_back(r.a);
        ctx->pool.push_back(r.b);
    }
    ctx->recs.clear();
    if (total_ms) *total_ms = ctx->prof_ms[kind];
    if (launches) *launches = ctx->prof_n[kind];
    ctx->prof_ms[kind] = 0.0;
    ctx->prof_n[kind] = 0;
    return TDGL_OK;
}

}  // extern "C"

// =============================================================================================
// Electrostatic field without any allocation (tdgl_elec_field_static).
//
// Some callers cannot call cudaMalloc: plug-ins whose host application owns every device byte
// through its own pool allocator, and real-time loops that may not block on the driver's
// allocator (cudaMalloc can synchronize the device).  For them this entry point computes the
// open-boundary field of a given P with every intermediate buffer (descriptor, work lists,
// twiddles, FP64 tensor temporaries, tensor spectrum, x- and y-spectra) carved out of one
// file-scope device array of fixed size.  The arithmetic is that of tdgl_get_field with the
// electrostatic term alone, but through the generic (any-length) row, y and z kernels, and the
// FP64 tensor spectrum is rebuilt on every call, since nothing survives between calls.
// =============================================================================================
namespace {

static __device__ __align__(256) unsigned char g_static_scratch[TDGL_STATIC_SCRATCH_BYTES];

const int kMaxDevices = 64;
void *g_static_ptr[kMaxDevices] = {nullptr};   // device address of g_static_scratch, per device
std::mutex g_static_setup;                      // guards the once-per-device set-up below

// Launch k<<<g, b, sm, st>>>(a...) and return the launch's own status (unlike cudaGetLastError,
// this neither reports nor clears an error that the caller left pending).
template <class... KA, class... A>
cudaError_t launch_status(void (*k)(KA...), dim3 g, dim3 b, size_t sm, cudaStream_t st, A &&...a) {
    std::tuple<KA...> t(std::forward<A>(a)...);
    void *args[sizeof...(KA) > 0 ? sizeof...(KA) : 1];
    std::apply([&](auto &...x) {
        int i = 0;
        ((args[i++] = static_cast<void *>(&x)), ...);
    }, t);
    return cudaLaunchKernel(reinterpret_cast<const void *>(k), g, b, args, sm, st);
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// radix plan without host twiddles (the table is written on the device)
Plan plan_only(int n, int tw_offset) {
    Plan p;
    memset(&p, 0, sizeof p);
    p.n = n;
    int r = n;
    const int rads[5] = {16, 8, 4, 3, 2};
    for (int i = 0; i < 5; ++i)
        while (r % rads[i] == 0 && r > 1) {
            p.rad[p.nrad++] = rads[i];
            r /= rads[i];
        }
    p.tw = tw_offset;
    return p;
}

struct StaticPlan {
    int nx, ny, nz, Mx, My, Mz, hx, Kx, kxp, kyh, kzh;
    int RB, KY, KZ, nrb, nky, nkz, n_rows, n_y, n_z;
    size_t o_desc, o_rows, o_y, o_z, o_tw, o_coef, o_mat, o_X, o_Y, o_Nhat, o_N, o_T1, o_T2, o_trig, o_slots, total;
    long ncell, n1, n2, n3;
};

StaticPlan static_plan(int nx, int ny, int nz) {
    StaticPlan q;
    memset(&q, 0, sizeof q);
    q.nx = nx; q.ny = ny; q.nz = nz;
    q.Mx = smooth_at_least(2 * nx - 1, true);
    q.My = smooth_at_least(2 * ny - 1, false);
    q.Mz = smooth_at_least(2 * nz - 1, false);
    q.hx = q.Mx / 2; q.Kx = q.hx + 1; q.kxp = (q.Kx + 3) & ~3; q.kyh = q.My / 2 + 1; q.kzh = q.Mz / 2 + 1;
    // chunking identical to build_items()
    q.RB = std::max(1, std::min(ny, std::max(1, 512 / nx)));
    q.KY = std::max(1, std::min(16, 73728 / (16 * (q.My + 1))));
    q.KZ = std::max(1, std::min(16, 102400 / (48 * (q.Mz + 1))));
    q.nrb = (ny + q.RB - 1) / q.RB;
    q.nky = (q.Kx + q.KY - 1) / q.KY;
    q.nkz = (q.Kx + q.KZ - 1) / q.KZ;
    q.n_rows = nz * q.nrb;
    q.n_y = 3 * nz * q.nky;
    q.n_z = q.My * q.nkz;
    q.ncell = (long)nx * ny * nz;
    q.n1 = (long)nz * ny * q.Kx;
    q.n2 = (long)nz * q.kyh * q.Kx;
    q.n3 = (long)q.kzh * q.kyh * q.Kx;
    size_t o = 0;
    auto take = [&](size_t bytes) { const size_t at = o; o = align256(o + bytes); return at; };
    q.o_desc = take(sizeof(SimDev));
    q.o_rows = take(sizeof(int4) * q.n_rows);
    q.o_y = take(sizeof(int4) * q.n_y);
    q.o_z = take(sizeof(int4) * q.n_z);
    q.o_tw = take(sizeof(float2) * (size_t)(q.hx + q.My + q.Mz + q.hx + 1));
    q.o_coef = take(sizeof(float) * MAXMAT * NCOEF);
    q.o_mat = take((size_t)q.ncell);
    q.o_X = take(sizeof(float2) * 3ull * nz * ny * q.kxp);
    q.o_Y = take(sizeof(float2) * 3ull * nz * q.My * q.kxp);
    q.o_Nhat = take(sizeof(float2) * 3ull * q.kzh * q.kyh * q.kxp);
    q.o_N = take(sizeof(double) * 6ull * q.ncell);
    q.o_T1 = take(sizeof(double) * 6ull * std::max(q.n1, q.n3));
    q.o_T2 = take(sizeof(double) * 6ull * std::max(q.n2, q.n3));
    q.o_trig = take(sizeof(double) * 2ull * (q.Mx + q.My + q.Mz));
    q.o_slots = take(64);
    q.total = o;
    return q;
}

// work lists of the three kernel families, written on the device (same order as build_items)
__global__ void k_static_items(int4 *rows, int4 *ys, int4 *zs, StaticPlan q) {
    const int n = q.n_rows + q.n_y + q.n_z;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (i < q.n_rows) {
            const int z = i / q.nrb, y0 = (i % q.nrb) * q.RB;
            rows[i] = make_int4(0, z, y0, min(q.RB, q.ny - y0));
        } else if (i < q.n_rows + q.n_y) {
            const int j = i - q.n_rows, cz = j / q.nky, k0 = (j % q.nky) * q.KY;
            ys[j] = make_int4(0, cz, k0, min(q.KY, q.Kx - k0));
        } else {
            const int j = i - q.n_rows - q.n_y, ky = j / q.nkz, k0 = (j % q.nkz) * q.KZ;
            zs[j] = make_int4(0, ky, k0, min(q.KZ, q.Kx - k0));
        }
    }
}

// the kernel descriptor's bytes, passed by value (kernel arguments are copied at launch) and stored
// on the device by one warp
struct DescBytes {
    unsigned long long w[(sizeof(SimDev) + 7) / 8];
};
__global__ void k_static_desc(unsigned long long *dst, DescBytes D) {
    if (blockIdx.x == 0)
        for (int i = threadIdx.x; i < (int)(sizeof(D.w) / 8); i += blockDim.x) dst[i] = D.w[i];
}

// FFT twiddles W_n^t (float32 from float64 sincospi) and the tensor transform's cos/sin tables
__global__ void k_static_tables(float2 *tw, double *trig, StaticPlan q) {
    const int ntw = q.hx + q.My + q.Mz + q.hx + 1;
    const int ntr = q.Mx + q.My + q.Mz;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ntw + ntr; i += gridDim.x * blockDim.x) {
        if (i < ntw) {
            int n, t;
            if (i < q.hx) { n = q.hx; t = i; }
            else if (i < q.hx + q.My) { n = q.My; t = i - q.hx; }
            else if (i < q.hx + q.My + q.Mz) { n = q.Mz; t = i - q.hx - q.My; }
            else { n = q.Mx; t = i - q.hx - q.My - q.Mz; }
            double s, c;
            sincospi(-2.0 * (double)t / (double)n, &s, &c);
            tw[i] = make_float2((float)c, (float)s);
        } else {
            const int j = i - ntw;
            int base, M, t;
            if (j < q.Mx) { base = 0; M = q.Mx; t = j; }
            else if (j < q.Mx + q.My) { base = 2 * q.Mx; M = q.My; t = j - q.Mx; }
            else { base = 2 * (q.Mx + q.My); M = q.Mz; t = j - q.Mx - q.My; }
            double s, c;
            sincospi(2.0 * (double)t / (double)M, &s, &c);
            trig[base + t] = c;
            trig[base + M + t] = s;
        }
    }
}

}  // namespace

extern "C" int tdgl_elec_field_static(int nx, int ny, int nz, double dx, double dy, double dz, double eps_b,
                                      const float *P, const uint8_t *mat, float *E, void *stream) {
    if (nx < 1 || ny < 1 || nz < 1 || nx > TDGL_MAX_DIM || ny > TDGL_MAX_DIM || nz > TDGL_MAX_DIM) return TDGL_EINVAL;
    if (!(dx > 0) || !(dy > 0) || !(dz > 0) || !std::isfinite(dx) || !std::isfinite(dy) || !std::isfinite(dz))
        return TDGL_EINVAL;
    if (!(eps_b > 0) || !std::isfinite(eps_b) || !P || !E) return TDGL_EINVAL;
    const StaticPlan q = static_plan(nx, ny, nz);
    if (q.total > (size_t)TDGL_STATIC_SCRATCH_BYTES) return TDGL_ETOOBIG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return TDGL_ECUDA;
    {
        // once per device, with that device current: device address of the scratch array and
        // the dynamic shared-memory limits of the kernels used below (serialized across threads)
        std::lock_guard<std::mutex> lock(g_static_setup);
        if (!g_static_ptr[dev]) {
            void *ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_static_scratch) != cudaSuccess || !ptr) return TDGL_ECUDA;
            const void *ks[5] = {reinterpret_cast<const void *>(k_rows<MODE_XFWD>),
                                 reinterpret_cast<const void *>(k_rows<MODE_FIELD>),
                                 reinterpret_cast<const void *>(k_yfwd), reinterpret_cast<const void *>(k_yinv),
                                 reinterpret_cast<const void *>(k_zconv)};
            for (const void *k : ks)
                if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem) != cudaSuccess)
                    return TDGL_ECUDA;
            g_static_ptr[dev] = ptr;
        }
    }
    unsigned char *base = static_cast<unsigned char *>(g_static_ptr[dev]);
    cudaStream_t st = (cudaStream_t)stream;
    SimDev D;
    memset(&D, 0, sizeof D);
    D.nx = nx; D.ny = ny; D.nz = nz; D.ncell = q.ncell;
    D.hx = q.hx; D.Kx = q.Kx; D.kxp = q.kxp; D.My = q.My; D.Mz = q.Mz; D.kyh = q.kyh; D.kzh = q.kzh;
    D.px = plan_only(q.hx, 0);
    D.py = plan_only(q.My, q.hx);
    D.pz = plan_only(q.Mz, q.hx + q.My);
    D.twr = q.hx + q.My + q.Mz;
    D.tw = reinterpret_cast<const float2 *>(base + q.o_tw);
    D.P[0] = D.P[1] = const_cast<float *>(P);          // read only in the modes used here
    D.mat = mat ? mat : reinterpret_cast<const uint8_t *>(base + q.o_mat);
    D.X = reinterpret_cast<float2 *>(base + q.o_X);
    D.Y = reinterpret_cast<float2 *>(base + q.o_Y);
    D.Nhat = reinterpret_cast<const float2 *>(base + q.o_Nhat);
    D.coef = reinterpret_cast<const float *>(base + q.o_coef);
    D.escale = (float)(-1.0 / (kEps0 * eps_b) / ((double)q.Mx * q.My * q.Mz));   // alpha_ref = P0 = 1
    D.pmax = 1e3f;
    D.terms = TERM_ELEC;
    D.maxdp = reinterpret_cast<unsigned *>(base + q.o_slots);
    D.flag = reinterpret_cast<int *>(base + q.o_slots + 16);
    D.energy = reinterpret_cast<double *>(base + q.o_slots + 32);
    D.out = E;
    D.out_scale = 1.0f;
    const double ell = std::min(dx, std::min(dy, dz));
    for (int a = 0; a < 3; ++a) {
        const double h = (a == 0 ? dx : (a == 1 ? dy : dz)) / ell;
        D.inv_d2[a] = (float)(1.0 / (h * h));
        D.inv_2d[a] = (float)(1.0 / (2.0 * h));
    }
    const SimDev *ddesc = reinterpret_cast<const SimDev *>(base + q.o_desc);
    int4 *rows = reinterpret_cast<int4 *>(base + q.o_rows);
    int4 *ys = reinterpret_cast<int4 *>(base + q.o_y);
    int4 *zs = reinterpret_cast<int4 *>(base + q.o_z);
    double *dN = reinterpret_cast<double *>(base + q.o_N);
    double *dT1 = reinterpret_cast<double *>(base + q.o_T1);
    double *dT2 = reinterpret_cast<double *>(base + q.o_T2);
    double *trig = reinterpret_cast<double *>(base + q.o_trig);
    FarRule rule;
    memset(&rule, 0, sizeof rule);
    const int ms[3] = {8, 6, 4};
    for (int k = 0; k < 3; ++k) {
        rule.m[k] = ms[k];
        gauss_legendre01(ms[k], rule.tau[k], rule.wt[k]);
    }
    if (cudaMemsetAsync(base + q.o_coef, 0, sizeof(float) * MAXMAT * NCOEF, st) != cudaSuccess) return TDGL_ECUDA;
    if (!mat && cudaMemsetAsync(base + q.o_mat, 1, (size_t)q.ncell, st) != cudaSuccess) return TDGL_ECUDA;
    const int ntab = q.hx + q.My + q.Mz + q.hx + 1 + q.Mx + q.My + q.Mz;
    SimDev *desc_dst = reinterpret_cast<SimDev *>(base + q.o_desc);
    DescBytes Db;
    memset(&Db, 0, sizeof Db);
    memcpy(&Db, &D, sizeof D);
    float2 *tw_dst = reinterpret_cast<float2 *>(base + q.o_tw);
    float2 *nhat_dst = reinterpret_cast<float2 *>(base + q.o_Nhat);
    const dim3 b256(256);
    // x forward, y/z convolution, x inverse into E (the generic kernels)
    const size_t sm_rows = 2ull * 3 * q.RB * (q.hx + 2) * sizeof(float2);
    const size_t sm_y = 2ull * q.KY * (q.My + 1) * sizeof(float2);
    const size_t sm_z = 2ull * 3 * q.KZ * (q.Mz + 1) * sizeof(float2);
    const cudaError_t es[] = {
        launch_status(k_static_desc, dim3(1), dim3(32), 0, st, reinterpret_cast<unsigned long long *>(desc_dst), Db),
        launch_status(k_static_items, dim3(grid_for(q.n_rows + q.n_y + q.n_z)), b256, 0, st, rows, ys, zs, q),
        launch_status(k_static_tables, dim3(grid_for(ntab)), b256, 0, st, tw_dst, trig, q),
        // tensor spectrum (FP64), lengths in units of the smallest cell edge
        launch_status(k_tensor_real, dim3(grid_for(q.ncell)), b256, 0, st, dN, nx, ny, nz, dx / ell, dy / ell,
                      dz / ell, 5.0, 16.0, 40.0, rule),
        launch_status(k_tensor_dft, dim3(grid_for(6 * q.n1)), b256, 0, st, dN, dT1, 0, nx, q.Kx, q.Mx, 1, nz * ny,
                      trig, trig + q.Mx),
        launch_status(k_tensor_dft, dim3(grid_for(6 * q.n2)), b256, 0, st, dT1, dT2, 1, ny, q.kyh, q.My, q.Kx, nz,
                      trig + 2 * q.Mx, trig + 2 * q.Mx + q.My),
        launch_status(k_tensor_dft, dim3(grid_for(6 * q.n3)), b256, 0, st, dT2, dT1, 2, nz, q.kzh, q.Mz,
                      q.kyh * q.Kx, 1, trig + 2 * (q.Mx + q.My), trig + 2 * (q.Mx + q.My) + q.Mz),
        launch_status(k_tensor_store, dim3(grid_for(3L * q.kzh * q.kyh * q.kxp)), b256, 0, st, dT1, nhat_dst,
                      (long)q.kzh * q.kyh, q.Kx, q.kxp),
        launch_status(k_rows<MODE_XFWD>, dim3(q.n_rows), dim3(NTHREADS), sm_rows, st, ddesc, rows, 0),
        launch_status(k_yfwd, dim3(q.n_y), dim3(NTHREADS), sm_y, st, ddesc, ys),
        launch_status(k_zconv, dim3(q.n_z), dim3(NTHREADS), sm_z, st, ddesc, zs),
        launch_status(k_yinv, dim3(q.n_y), dim3(NTHREADS), sm_y, st, ddesc, ys),
        launch_status(k_rows<MODE_FIELD>, dim3(q.n_rows), dim3(NTHREADS), sm_rows, st, ddesc, rows, 0)};
    for (cudaError_t e : es)
        if (e != cudaSuccess) return TDGL_ECUDA;
    return TDGL_OK;
}
