// Row kernel with a shared-memory tile and register x-transforms (x complex length HX).
//
// A block owns TY consecutive x-rows (y0 .. y0+TY-1) of one plane z.  It stages the material ids of
// planes z-1, z, z+1 and P of plane z, rows y0-1 .. y0+TY, all x, in shared memory; P of planes z-1
// and z+1 comes from global memory through the L1 cache.  That covers every neighbour the discrete
// Eq. 4 needs (faces, and the edge cells of the cross terms), with
// cells outside the grid stored as vacuum.  Per mode:
//   STEP    x-inverse of the field spectrum (C2R) -> E_el rows; Landau (Eq. 3), gradient (Eq. 4),
//           E_ext (Eq. 7); forward Euler update (Eq. 1); x-forward (R2C) of the new rows.
//   FIELD   the same field, written out instead of the update.
//   ENERGY  energy densities (float32 per cell, float64 sums) of Eqs. 3-7.
//   XFWD    x-forward of the current rows only.
// Line (c, r) of the x-transforms is held by T = HX/E threads, thread t holding elements
// t + T m; the exchange buffer is [line][pos] padded by one slot in 16.
#pragma once
#include "fft_reg.cuh"
#include "kernels.cuh"

namespace tdgl {

// rows per block (TYC) and threads per block for the x-transform length HX (row length NX = HX)
template <int HX> __host__ __device__ constexpr int xrows_tile() {
    return (192 / (3 * rf::threads_per_line<HX>())) < 16 ? (192 / (3 * rf::threads_per_line<HX>())) : 16;
}
// (at least 192: for short rows the threads past the transform lines still share the staging and
// the cells)
template <int HX> __host__ __device__ constexpr int xrows_threads() {
    return ((3 * xrows_tile<HX>() * rf::threads_per_line<HX>()) + 31) / 32 * 32 > 192
               ? ((3 * xrows_tile<HX>() * rf::threads_per_line<HX>()) + 31) / 32 * 32
               : 192;
}
template <int HX> __host__ __device__ constexpr int xrows_ldp() { return HX + HX / 16 + 1; }
// floats of the region shared by the centre-plane P tile and the x-transform exchange (multiple of 4)
template <int HX> __host__ __device__ constexpr int xrows_region() {
    constexpr int tile = 3 * (xrows_tile<HX>() + 2) * HX;
    constexpr int exch = 2 * (xrows_threads<HX>() / rf::threads_per_line<HX>()) * xrows_ldp<HX>();
    return ((tile > exch ? tile : exch) + 3) & ~3;
}
// dynamic shared memory of k_xrows (bytes): shared region, E / new-P rows, material tile
template <int HX> __host__ __device__ constexpr size_t xrows_smem() {
    return ((sizeof(float) * ((size_t)xrows_region<HX>() + 3ull * xrows_tile<HX>() * HX) +
             3ull * (xrows_tile<HX>() + 2) * HX) + 15) & ~(size_t)15;
}

// Neighbourhood of a block's cells: materials of planes z-1, z, z+1 (rows y0-1 .. y0+TY, all x,
// out-of-grid cells vacuum) and P of the centre plane in shared memory; P of planes z-1 and z+1
// is read through the L1 cache from global memory.  Every caller reads P only at material cells
// (checked on the material tile first), which are inside the grid.
template <int NX, int TYH>
struct TileView {
    const float *P;       // centre plane [3 comps][TYH rows][NX], shared memory
    const float *G;       // the sim's P (global), component stride ncell
    long ncell;
    long row0[2];         // index of (plane z-1 / z+1, row y0-1, x 0) in one component of G
    const uint8_t *M;     // [3 planes][TYH][NX]
    __device__ __forceinline__ int m(int pz, int py, int x) const {
        return (unsigned)x < (unsigned)NX ? (int)M[(pz * TYH + py) * NX + x] : 0;
    }
    __device__ __forceinline__ float p(int c, int pz, int py, int x) const {
        if (pz == 1) return P[(c * TYH + py) * NX + x];
        return __ldg(G + c * ncell + row0[pz >> 1] + py * NX + x);
    }
};

__device__ __forceinline__ void nbr(int d, int s, int &pz, int &py, int &x) {
    if (d == 0) x += s; else if (d == 1) py += s; else pz += s;
}

// D_d P_f at a material tile cell, mirror ghosts at non-material neighbours
template <class TV>
__device__ __forceinline__ float tcentral(const TV &V, const SimDev &S, int pz, int py, int x, int d, int f) {
    const float q0 = V.p(f, pz, py, x);
    int az = pz, ay = py, ax = x, bz = pz, by = py, bx = x;
    nbr(d, 1, az, ay, ax);
    nbr(d, -1, bz, by, bx);
    const float qp = V.m(az, ay, ax) ? V.p(f, az, ay, ax) : q0;
    const float qm = V.m(bz, by, bx) ? V.p(f, bz, by, bx) : q0;
    return (qp - qm) * S.inv_2d[d];
}

// cross-term fluxes attached to direction d at a material tile cell (see cross_fluxes)
template <class TV>
__device__ __forceinline__ void tfluxes(const TV &V, const SimDev &S, const float *coef, int pz, int py, int x,
                                        int m, int d, float &Sd, float *T) {
    const float *c = coef + m * NCOEF;
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 3; ++j)
        if (j != d) s += tcentral(V, S, pz, py, x, j, j);
    Sd = c[10] * s;
#pragma unroll
    for (int i = 0; i < 3; ++i) T[i] = (i != d) ? c[11] * tcentral(V, S, pz, py, x, i, d) : 0.f;
}

// gradient field of the discrete Eq. 4 at centre-plane tile cell (1, py, x) of material ma
template <class TV>
__device__ __forceinline__ void tgrad_field(const TV &V, const SimDev &S, const float *coef, int py, int x,
                                            int ma, const float *pa, float *h, bool known_bulk) {
    const float *ca = coef + ma * NCOEF;
    // Bulk cells (the 6 face and, with cross terms, the 12 edge neighbours all of material ma):
    // no ghost rule applies and the coefficients are uniform, so the discrete field below reduces
    // exactly to G (P(+) + P(-) - 2P) / dx^2 per face pair plus (G12 + G44 - G'44) times the
    // four-corner mixed differences d_e d_f P_f.  known_bulk: the caller has established it.
    bool bulk = known_bulk || (V.m(1, py, x - 1) == ma && V.m(1, py, x + 1) == ma && V.m(1, py - 1, x) == ma &&
                               V.m(1, py + 1, x) == ma && V.m(0, py, x) == ma && V.m(2, py, x) == ma);
    if (bulk && !known_bulk && S.has_cross)
        bulk = V.m(1, py - 1, x - 1) == ma && V.m(1, py - 1, x + 1) == ma && V.m(1, py + 1, x - 1) == ma &&
               V.m(1, py + 1, x + 1) == ma && V.m(0, py, x - 1) == ma && V.m(0, py, x + 1) == ma &&
               V.m(2, py, x - 1) == ma && V.m(2, py, x + 1) == ma && V.m(0, py - 1, x) == ma &&
               V.m(0, py + 1, x) == ma && V.m(2, py - 1, x) == ma && V.m(2, py + 1, x) == ma;
    if (bulk) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const float lx = V.p(i, 1, py, x - 1) + V.p(i, 1, py, x + 1) - 2.f * pa[i];
            const float ly = V.p(i, 1, py - 1, x) + V.p(i, 1, py + 1, x) - 2.f * pa[i];
            const float lz = V.p(i, 0, py, x) + V.p(i, 2, py, x) - 2.f * pa[i];
            const float gx = (i == 0) ? ca[8] : ca[9], gy = (i == 1) ? ca[8] : ca[9], gz = (i == 2) ? ca[8] : ca[9];
            h[i] = fmaf(gx * S.inv_d2[0], lx, fmaf(gy * S.inv_d2[1], ly, fmaf(gz * S.inv_d2[2], lz, h[i])));
        }
        if (S.has_cross) {
            const float C = ca[10] + ca[11];
            const float wxy = C * S.inv_2d[0] * S.inv_2d[1], wxz = C * S.inv_2d[0] * S.inv_2d[2],
                        wyz = C * S.inv_2d[1] * S.inv_2d[2];
            auto cxy = [&](int f) {   // (x+,y+) - (x+,y-) - (x-,y+) + (x-,y-)
                return V.p(f, 1, py + 1, x + 1) - V.p(f, 1, py - 1, x + 1) - V.p(f, 1, py + 1, x - 1) +
                       V.p(f, 1, py - 1, x - 1);
            };
            auto cxz = [&](int f) {
                return V.p(f, 2, py, x + 1) - V.p(f, 0, py, x + 1) - V.p(f, 2, py, x - 1) + V.p(f, 0, py, x - 1);
            };
            auto cyz = [&](int f) {
                return V.p(f, 2, py + 1, x) - V.p(f, 0, py + 1, x) - V.p(f, 2, py - 1, x) + V.p(f, 0, py - 1, x);
            };
            h[0] = fmaf(wxy, cxy(1), fmaf(wxz, cxz(2), h[0]));
            h[1] = fmaf(wxy, cxy(0), fmaf(wyz, cyz(2), h[1]));
            h[2] = fmaf(wxz, cxz(0), fmaf(wyz, cyz(1), h[2]));
        }
        return;
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
#pragma unroll
        for (int s = -1; s <= 1; s += 2) {
            int nz_ = 1, ny_ = py, nx_ = x;
            nbr(d, s, nz_, ny_, nx_);
            const int mb = V.m(nz_, ny_, nx_);
            if (!mb) continue;
            const float *cb = coef + mb * NCOEF;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const float g = 0.5f * ((i == d) ? ca[8] + cb[8] : ca[9] + cb[9]) * S.inv_d2[d];
                h[i] = fmaf(g, V.p(i, nz_, ny_, nx_) - pa[i], h[i]);
            }
        }
    }
    if (!S.has_cross) return;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        float Sa, Ta[3], Sp, Tp[3], Sm, Tm[3];
        tfluxes(V, S, coef, 1, py, x, ma, d, Sa, Ta);
        int az = 1, ay = py, ax = x, bz = 1, by = py, bx = x;
        nbr(d, 1, az, ay, ax);
        nbr(d, -1, bz, by, bx);
        const int mp = V.m(az, ay, ax), mm = V.m(bz, by, bx);
        if (mp) tfluxes(V, S, coef, az, ay, ax, mp, d, Sp, Tp);
        else { Sp = -Sa; Tp[0] = -Ta[0]; Tp[1] = -Ta[1]; Tp[2] = -Ta[2]; }
        if (mm) tfluxes(V, S, coef, bz, by, bx, mm, d, Sm, Tm);
        else { Sm = -Sa; Tm[0] = -Ta[0]; Tm[1] = -Ta[1]; Tm[2] = -Ta[2]; }
        const float w = S.inv_2d[d];
        h[d] = fmaf(Sp - Sm, w, h[d]);
#pragma unroll
        for (int i = 0; i < 3; ++i)
            if (i != d) h[i] = fmaf(Tp[i] - Tm[i], w, h[i]);
    }
}

// gradient energy density at centre-plane cell: faces towards +x, +y, +z and the cross terms
template <class TV>
__device__ __forceinline__ float tgrad_energy(const TV &V, const SimDev &S, const float *coef, int py, int x,
                                              int ma, const float *pa) {
    const float *ca = coef + ma * NCOEF;
    float e = 0.f;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        int nz_ = 1, ny_ = py, nx_ = x;
        nbr(d, 1, nz_, ny_, nx_);
        const int mb = V.m(nz_, ny_, nx_);
        if (!mb) continue;
        const float *cb = coef + mb * NCOEF;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const float g = 0.5f * ((i == d) ? ca[8] + cb[8] : ca[9] + cb[9]) * S.inv_d2[d];
            const float df = V.p(i, nz_, ny_, nx_) - pa[i];
            e = fmaf(0.5f * g * df, df, e);
        }
    }
    if (S.has_cross) {
        float D[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int d = 0; d < 3; ++d) D[i][d] = tcentral(V, S, 1, py, x, d, i);
        e += ca[10] * (D[0][0] * D[1][1] + D[1][1] * D[2][2] + D[2][2] * D[0][0]) +
             ca[11] * (D[0][1] * D[1][0] + D[1][2] * D[2][1] + D[0][2] * D[2][0]);
    }
    return e;
}

template <int MODE, int HX>
__global__ void __launch_bounds__(192) k_xrows(const SimDev *__restrict__ sims, const int4 *__restrict__ items,
                                               int istep) {
    constexpr int E = rf::Cfg<HX>::E, T = HX / E, LDP = xrows_ldp<HX>();
    constexpr int nx = HX, TYmax = xrows_tile<HX>(), TYH = TYmax + 2, nthr = xrows_threads<HX>();
    extern __shared__ float4 smem4[];
    __shared__ float s_coef[MAXMAT * NCOEF];
    __shared__ float2 s_tw[HX];          // W_HX^t for the complex transform
    __shared__ float2 s_twr[HX + 1];     // W_Mx^k for the real pre/post-processing
    __shared__ double s_red[8];
    __shared__ unsigned s_max;
    const int4 it = items[blockIdx.x];
    const SimDev &S = sims[it.x];
    const int z = it.y, y0 = it.z, TY = it.w;     // TY rows of this block (<= tile)
    const int ny = S.ny, nz = S.nz;
    const int tid = threadIdx.x;
    // layout (xrows_smem): region R = max(P tile [3][3][TYH][nx] floats, x-transform exchange
    // [nthr/T][LDP] float2; the exchange is only live while the tile is not), then the E / new-P
    // rows [3][TYmax][nx] and the material tile [3][TYH][nx]
    float *Pt = reinterpret_cast<float *>(smem4);
    float2 *X2 = reinterpret_cast<float2 *>(smem4);
    constexpr int rf_ = xrows_region<HX>();                     // floats, multiple of 4
    float *Eb = Pt + rf_;
    uint8_t *Mt = reinterpret_cast<uint8_t *>(Eb + 3 * TYmax * nx);
    const int parity = istep & 1;      // istep: step index within the call
    // HEUN2 evaluates the field on the predictor (other buffer) and updates P in place
    const float *Pc = (MODE == MODE_HEUN2) ? S.P[parity ^ 1] : S.P[parity];
    float *Pn = (MODE == MODE_HEUN2) ? S.P[parity] : S.P[parity ^ 1];
    const bool elec = (S.terms & TERM_ELEC) != 0;
    float eext[3];
    ext_field(S, istep, eext);
    for (int i = tid; i < MAXMAT * NCOEF; i += nthr) s_coef[i] = S.coef[i];
    for (int i = tid; i < HX; i += nthr) s_tw[i] = S.tw[S.px.tw + i];
    for (int i = tid; i <= HX; i += nthr) s_twr[i] = S.tw[S.twr + i];
    if (tid == 0) s_max = 0u;
    // ---- x-inverse of the field spectrum: line l = c*TY + r held by T threads
    const int line = tid / T, t = tid % T;
    const int nlines = 3 * TYmax;
    const int lc = line / TYmax, lr = line % TYmax;
    const bool lok = line < nlines && lr < TY;
    auto xidx = [&](int pos) { return line * LDP + pos + (pos >> 4); };
    __syncthreads();   // twiddle and coefficient tables
    if (MODE != MODE_XFWD && elec) {
        float2 v[E];
        const float2 *row = S.X + (((long)lc * nz + z) * ny + y0 + lr) * S.kxp;
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int k = t + T * m;
            float2 a = make_float2(0.f, 0.f), b = make_float2(0.f, 0.f);
            if (lok) { a = row[k]; b = cconj(row[HX - k]); }
            const float2 w = cconj(s_twr[k]);               // W^{-k}
            const float2 d = cmul(csub(a, b), w);
            v[m] = make_float2(a.x + b.x - d.y, a.y + b.y + d.x);
        }
        rf::fft<rf::Cfg<HX>, true>(v, t, X2, xidx, s_tw);
        if (lok) {
#pragma unroll
            for (int i = 0; i < E; ++i) {
                const int j = rf::final_pos<rf::Cfg<HX>>(t, i);
                const int x0 = 2 * j;
                float *er = Eb + (lc * TYmax + lr) * nx;
                if (rf::kept_out<rf::Cfg<HX>>(i) && x0 < nx) er[x0] = v[i].x;
                if (rf::kept_out<rf::Cfg<HX>>(i) && x0 + 1 < nx) er[x0 + 1] = v[i].y;
            }
        }
        __syncthreads();
    }
    // ---- stage the P / material tile (cells outside the grid: vacuum, P = 0); note whether the
    // whole tile (all planes and halo rows the cells read) is one material inside the grid: then
    // every cell with 0 < x < nx - 1 is a bulk cell of the discrete Eq. 4
    bool uniform = MODE != MODE_XFWD;
    const unsigned m0x4 = 0x01010101u * (unsigned)__ldg(S.mat + ((long)z * ny + y0) * nx);
    {
        const int planes = (MODE == MODE_XFWD) ? 1 : 3;
        const int nrow = planes * TYH;
        static_assert(nx % 4 == 0, "row length must be a multiple of 4");
        for (int w = tid; w < nrow * (nx / 4); w += nthr) {
            const int q = w % (nx / 4), rr = w / (nx / 4);
            const int py = rr % TYH;
            const int pz = (MODE == MODE_XFWD) ? 1 : rr / TYH;
            const int gy = y0 - 1 + py, gz = z - 1 + pz;
            const bool in = (unsigned)gy < (unsigned)ny && (unsigned)gz < (unsigned)nz && py <= TY + 1;
            const unsigned v = in ? __ldg(reinterpret_cast<const unsigned *>(S.mat + ((long)gz * ny + gy) * nx) + q) : 0u;
            reinterpret_cast<unsigned *>(Mt + (pz * TYH + py) * nx)[q] = v;
            // rows past this block's TY + 2 are never read; every other word must be m0 in each byte
            if (py <= TY + 1 && v != m0x4) uniform = false;
        }
        // P: the centre plane only (planes z +- 1 are read from global memory by the cells)
        if ((nx & 3) == 0) {   // rows of nx floats: 16-byte vector copies
            const int nq = nx >> 2;
            for (int w = tid; w < 3 * TYH * nq; w += nthr) {
                const int q = w % nq, rr = w / nq;
                const int py = rr % TYH, c = rr / TYH;
                const int gy = y0 - 1 + py;
                const bool in = (unsigned)gy < (unsigned)ny && py <= TY + 1;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (in) v = __ldg(reinterpret_cast<const float4 *>(Pc + c * S.ncell + ((long)z * ny + gy) * nx) + q);
                reinterpret_cast<float4 *>(Pt + (c * TYH + py) * nx)[q] = v;
            }
        } else {
            for (int w = tid; w < 3 * TYH * nx; w += nthr) {
                const int x = w % nx, rr = w / nx;
                const int py = rr % TYH, c = rr / TYH;
                const int gy = y0 - 1 + py;
                const bool in = (unsigned)gy < (unsigned)ny && py <= TY + 1;
                Pt[(c * TYH + py) * nx + x] = in ? __ldg(&Pc[c * S.ncell + ((long)z * ny + gy) * nx + x]) : 0.f;
            }
        }
    }
    const bool tile_bulk = __syncthreads_and(uniform && m0x4 != 0u) != 0;
    // ---- cells
    const TileView<nx, TYH> V{Pt, Pc, S.ncell, {((long)(z - 1) * ny + y0 - 1) * nx, ((long)(z + 1) * ny + y0 - 1) * nx}, Mt};
    float lmax = 0.f;
    bool bad = false;
    double e_land = 0.0, e_grad = 0.0, e_elec = 0.0, e_ext = 0.0;
    if (MODE != MODE_XFWD) {
        for (int w = tid; w < TY * nx; w += nthr) {
            const int r = w / nx, x = w - r * nx;
            const int py = r + 1;
            const long id = ((long)z * ny + y0 + r) * nx + x;
            const int m = V.m(1, py, x);
            if (m == 0) {
                if (mode_updates(MODE)) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) { Pn[c * S.ncell + id] = 0.f; Eb[(c * TYmax + r) * nx + x] = 0.f; }
                } else if (MODE == MODE_FIELD) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) S.out[c * S.ncell + id] = 0.f;
                } else if (MODE == MODE_DERIV) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) S.hbuf[c * S.ncell + id] = 0.f;
                }
                continue;
            }
            float p[3], h[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int c = 0; c < 3; ++c) p[c] = V.p(c, 1, py, x);
            const float *cm = s_coef + m * NCOEF;
            if (MODE == MODE_ENERGY) {
                if (S.terms & TERM_LANDAU) {
                    const float x2 = p[0] * p[0], y2 = p[1] * p[1], z2 = p[2] * p[2];
                    const float f = cm[0] * x2 + cm[1] * y2 + cm[2] * z2 + cm[3] * (x2 * x2 + y2 * y2 + z2 * z2) +
                                    cm[4] * (x2 * y2 + y2 * z2 + z2 * x2) +
                                    cm[5] * (x2 * x2 * x2 + y2 * y2 * y2 + z2 * z2 * z2) +
                                    cm[6] * (x2 * x2 * (y2 + z2) + y2 * y2 * (x2 + z2) + z2 * z2 * (x2 + y2)) +
                                    cm[7] * x2 * y2 * z2;
                    e_land += (double)f;
                }
                if (S.terms & TERM_GRAD) e_grad += (double)tgrad_energy(V, S, s_coef, py, x, m, p);
                float el = 0.f, ex = 0.f;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    if (elec) el = fmaf(-0.5f * Eb[(c * TYmax + r) * nx + x], p[c], el);
                    if (S.terms & TERM_EXT) ex = fmaf(-eext[c], p[c], ex);
                }
                e_elec += (double)el;
                e_ext += (double)ex;
                continue;
            }
            if (S.terms & TERM_LANDAU) landau_field(p, cm, h);
            if (S.terms & TERM_GRAD) tgrad_field(V, S, s_coef, py, x, m, p, h, tile_bulk && x > 0 && x < nx - 1);
            if (elec) {
#pragma unroll
                for (int c = 0; c < 3; ++c) h[c] += Eb[(c * TYmax + r) * nx + x];
            }
            if (S.terms & TERM_EXT) {
#pragma unroll
                for (int c = 0; c < 3; ++c) h[c] += eext[c];
            }
            if (MODE == MODE_FIELD) {
#pragma unroll
                for (int c = 0; c < 3; ++c) S.out[c * S.ncell + id] = h[c] * S.out_scale;
                continue;
            }
            if (MODE == MODE_DERIV) {   // dP/dt of Eq. 1 (L = 1, normalized) for a multi-stage integrator
#pragma unroll
                for (int c = 0; c < 3; ++c) S.hbuf[c * S.ncell + id] = h[c];
                continue;
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float pn, p0 = p[c];
                if (MODE == MODE_HEUN2) {
                    p0 = Pn[c * S.ncell + id];
                    pn = fmaf(0.5f * S.dt, S.hbuf[c * S.ncell + id] + h[c], p0);
                } else {
                    pn = fmaf(S.dt, h[c], p0);
                    if (MODE == MODE_HEUN1) S.hbuf[c * S.ncell + id] = h[c];
                }
                if (MODE != MODE_HEUN1) lmax = fmaxf(lmax, fabsf(pn - p0));
                bad |= !(fabsf(pn) <= S.pmax);
                Pn[c * S.ncell + id] = pn;
                Eb[(c * TYmax + r) * nx + x] = pn;      // the cell's own slot: E read above, new P kept
            }
        }
    }
    if (MODE == MODE_ENERGY) {
        double v;
        v = block_sum(e_land, s_red); if (tid == 0) atomicAdd(&S.energy[0], v);
        v = block_sum(e_grad, s_red); if (tid == 0) atomicAdd(&S.energy[1], v);
        v = block_sum(e_elec, s_red); if (tid == 0) atomicAdd(&S.energy[2], v);
        v = block_sum(e_ext, s_red); if (tid == 0) atomicAdd(&S.energy[3], v);
        return;
    }
    if (MODE == MODE_FIELD || MODE == MODE_DERIV) return;
    if (mode_updates(MODE)) {
        for (int o = 16; o > 0; o >>= 1) lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
        if ((tid & 31) == 0) atomicMax(&s_max, __float_as_uint(lmax));
        if (bad) atomicOr(S.flag, 1);
        __syncthreads();
        if (tid == 0) atomicMax(S.maxdp, s_max);
    }
    if (!elec) return;
    __syncthreads();
    // ---- x-forward of the new (STEP) or current (XFWD) rows: z_j = (x_2j, x_2j+1), zero padded
    {
        float2 v[E];
        const float *src = (MODE == MODE_XFWD) ? Pt + (lc * TYH + lr + 1) * nx : Eb + (lc * TYmax + lr) * nx;
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int j = t + T * m;
            const int x0 = 2 * j;
            const bool in = rf::padded_in<rf::Cfg<HX>>(m) && lok;   // x0 = 2j, j >= HX/2: padding
            v[m] = make_float2((in && x0 < nx) ? src[x0] : 0.f, (in && x0 + 1 < nx) ? src[x0 + 1] : 0.f);
        }
        __syncthreads();   // the exchange below reuses the tile's memory
        rf::fft<rf::Cfg<HX>, false>(v, t, X2, xidx, s_tw);
        // Hermitian half-spectrum from the packed transform: needs Z_k and Z_{HX-k}
#pragma unroll
        for (int i = 0; i < E; ++i) X2[xidx(rf::final_pos<rf::Cfg<HX>>(t, i))] = v[i];
        __syncthreads();
        if (lok) {
            float2 *row = S.X + (((long)lc * nz + z) * ny + y0 + lr) * S.kxp;
            for (int k = t; k <= HX; k += T) {
                const float2 a = X2[xidx(k == HX ? 0 : k)];
                const float2 b = cconj(X2[xidx(k == 0 ? 0 : HX - k)]);
                const float2 d = cmul(csub(a, b), s_twr[k]);
                row[k] = make_float2(0.5f * (a.x + b.x + d.y), 0.5f * (a.y + b.y - d.x));
            }
        }
    }
}

}  // namespace tdgl
