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
#include <type_traits>

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
// (checked on the material tile first), which are inside the grid.  Tile rows are LX apart in
// shared memory (the x half-length); a grid row holds nx <= LX cells.
template <int LX, int TYH, bool SHORT>
struct TileView {
    const float *P;       // centre plane [3 comps][TYH rows][LX], shared memory
    const float *G;       // the sim's P (global), component stride ncell
    long ncell;
    long row0[2];         // index of (plane z-1 / z+1, row y0-1, x 0) in one component of G
    const uint8_t *M;     // [3 planes][TYH][LX]
    int nxr;              // cells per row when SHORT (else LX)
    __device__ __forceinline__ int nx() const {
        if constexpr (SHORT) return nxr;
        else return LX;
    }
    __device__ __forceinline__ int m(int pz, int py, int x) const {
        return (unsigned)x < (unsigned)nx() ? (int)M[(pz * TYH + py) * LX + x] : 0;
    }
    __device__ __forceinline__ float p(int c, int pz, int py, int x) const {
        if (pz == 1) return P[(c * TYH + py) * LX + x];
        return __ldg(G + c * ncell + row0[pz >> 1] + py * nx() + x);
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
            // (P(z+1) - P(z-1)) at x+1 minus the same at x-1, and the y analogue
            auto cxz = [&](int f) {
                return (V.p(f, 2, py, x + 1) - V.p(f, 0, py, x + 1)) - (V.p(f, 2, py, x - 1) - V.p(f, 0, py, x - 1));
            };
            auto cyz = [&](int f) {
                return (V.p(f, 2, py + 1, x) - V.p(f, 0, py + 1, x)) - (V.p(f, 2, py - 1, x) - V.p(f, 0, py - 1, x));
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

template <int MODE, int HX, bool SHORT = false>
__global__ void __launch_bounds__(192, 4) k_xrows(const SimDev *__restrict__ sims, const int4 *__restrict__ items,
                                               int istep) {
    constexpr int E = rf::Cfg<HX>::E, T = HX / E, LDP = xrows_ldp<HX>();
    // LX: row stride of the shared tiles (the x half-length); nx: cells per grid row, LX itself
    // unless SHORT (then nx <= LX, a multiple of 4; the x transforms zero-pad the rest of the row)
    constexpr int LX = HX, TYmax = xrows_tile<HX>(), TYH = TYmax + 2, nthr = xrows_threads<HX>();
    extern __shared__ float4 smem4[];
    __shared__ float s_coef[MAXMAT * NCOEF];
    __shared__ float2 s_tw[HX];          // W_HX^t for the complex transform
    __shared__ float2 s_twr[HX + 1];     // W_Mx^k for the real pre/post-processing
    __shared__ double s_red[8];
    __shared__ unsigned s_max;
    __shared__ unsigned s_bad;           // bit py: tile row py is not all material m0 (or outside)
    __shared__ unsigned s_bad2;          // bit py: tile row py has a cell inside the grid that is not m0
    __shared__ unsigned char s_rowidx[2][16];   // the block's bulk rows, then its other rows, in order
    const int4 it = items[blockIdx.x];
    const SimDev &S = sims[it.x];
    if (S.skip) return;   // a batch member that has left the relaxation
    const int z = it.y, y0 = it.z, TY = it.w;     // TY rows of this block (<= tile)
    const int nx = [&] {
        if constexpr (SHORT) return S.nx;
        else return LX;
    }();
    const int ny = S.ny, nz = S.nz;
    const int tid = threadIdx.x;
    // layout (xrows_smem): region R = max(P tile [3][3][TYH][LX] floats, x-transform exchange
    // [nthr/T][LDP] float2; the exchange is only live while the tile is not), then the E / new-P
    // rows [3][TYmax][LX] and the material tile [3][TYH][LX]
    float *Pt = reinterpret_cast<float *>(smem4);
    float2 *X2 = reinterpret_cast<float2 *>(smem4);
    constexpr int rf_ = xrows_region<HX>();                     // floats, multiple of 4
    float *Eb = Pt + rf_;
    uint8_t *Mt = reinterpret_cast<uint8_t *>(Eb + 3 * TYmax * LX);
    const int parity = istep & 1;      // istep: step index within the call
    // HEUN2 evaluates the field on the predictor (other buffer) and updates P in place
    const float *Pc = (MODE == MODE_HEUN2) ? S.P[parity ^ 1] : S.P[parity];
    float *Pn = (MODE == MODE_HEUN2) ? S.P[parity] : S.P[parity ^ 1];
    const bool elec = (S.terms & TERM_ELEC) != 0;
    float eext[3];
    ext_field(S, istep, eext);
    // material tile of planes z-1, z, z+1 (XFWD: z only), rows y0-1 .. y0+TY: 4-byte asynchronous
    // copies issued now, zero (vacuum) outside the grid, waited for before the cells
    const unsigned m0x4 = 0x01010101u * (unsigned)__ldg(S.mat + ((long)z * ny + y0) * nx);
    const int mrow = ((MODE == MODE_XFWD) ? 1 : 3) * TYH;
    static_assert(LX % 4 == 0, "tile rows must be a multiple of 4 long");
    for (int w = tid; w < mrow * (nx / 4); w += nthr) {
        const int q = w % (nx / 4), rr = w / (nx / 4);
        const int py = rr % TYH;
        const int pz = (MODE == MODE_XFWD) ? 1 : rr / TYH;
        const int gy = y0 - 1 + py, gz = z - 1 + pz;
        const bool in = (unsigned)gy < (unsigned)ny && (unsigned)gz < (unsigned)nz && py <= TY + 1;
        const uint8_t *g = in ? S.mat + ((long)gz * ny + gy) * nx + 4 * q : S.mat;
        const unsigned dst = (unsigned)__cvta_generic_to_shared(Mt + (pz * TYH + py) * LX + 4 * q);
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(dst), "l"(g), "r"(in ? 4 : 0));
    }
    asm volatile("cp.async.commit_group;\n" ::);
    for (int i = tid; i < MAXMAT * NCOEF; i += nthr) s_coef[i] = S.coef[i];
    for (int i = tid; i < HX; i += nthr) s_tw[i] = S.tw[S.px.tw + i];
    for (int i = tid; i <= HX; i += nthr) s_twr[i] = S.tw[S.twr + i];
    if (tid == 0) { s_max = 0u; s_bad = 0u; s_bad2 = 0u; }
    // ---- x-inverse of the field spectrum: line l = c*TY + r held by T threads
    const int line = tid / T, t = tid % T;
    const int nlines = 3 * TYmax;
    const int lc = line / TYmax, lr = line % TYmax;
    const bool lok = line < nlines && lr < TY;
    auto xidx = [&](int pos) { return line * LDP + pos + (pos >> 4); };
    // the field spectrum's rows are loaded before the table barrier, so that both latencies overlap
    float2 xa[(MODE != MODE_XFWD) ? E : 1], xb[(MODE != MODE_XFWD) ? E : 1];
    if (MODE != MODE_XFWD && elec) {
        const float2 *row = S.X + (((long)lc * nz + z) * ny + y0 + lr) * S.kxp;
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int k = t + T * m;
            xa[m] = lok ? row[k] : make_float2(0.f, 0.f);
            xb[m] = lok ? cconj(row[HX - k]) : make_float2(0.f, 0.f);
        }
    }
    __syncthreads();   // twiddle and coefficient tables
    if (MODE != MODE_XFWD && elec) {
        float2 v[E];
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int k = t + T * m;
            const float2 a = xa[m], b = xb[m];
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
                float *er = Eb + (lc * TYmax + lr) * LX;
                if (rf::kept_out<rf::Cfg<HX>>(i) && x0 < nx) er[x0] = v[i].x;
                if (rf::kept_out<rf::Cfg<HX>>(i) && x0 + 1 < nx) er[x0 + 1] = v[i].y;
            }
        }
        __syncthreads();
    }
    // ---- stage the P / material tile (cells outside the grid: vacuum, P = 0); note which tile rows
    // are, in all three planes, inside the grid and of one material m0: a cell with 0 < x < nx - 1
    // whose own row and the rows on either side are all such rows is a bulk cell of the discrete
    // Eq. 4 (all 18 neighbours inside the grid and of its own material)
    {
        // the material tile has arrived (its copies were issued at the start); rows past this
        // block's TY + 2 are never read; every other word must be m0 in each byte
        asm volatile("cp.async.wait_group 0;\n" ::);
        for (int w = tid; w < mrow * (nx / 4); w += nthr) {
            const int q = w % (nx / 4), rr = w / (nx / 4);
            const int py = rr % TYH;
            const int pz = (MODE == MODE_XFWD) ? 1 : rr / TYH;
            const unsigned v = reinterpret_cast<const unsigned *>(Mt + (pz * TYH + py) * LX)[q];
            if (MODE != MODE_XFWD && py <= TY + 1 && v != m0x4) {
                const int gy = y0 - 1 + py, gz = z - 1 + pz;
                atomicOr(&s_bad, 1u << py);
                if ((unsigned)gy < (unsigned)ny && (unsigned)gz < (unsigned)nz) atomicOr(&s_bad2, 1u << py);
            }
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
                reinterpret_cast<float4 *>(Pt + (c * TYH + py) * LX)[q] = v;
            }
        } else {
            for (int w = tid; w < 3 * TYH * nx; w += nthr) {
                const int x = w % nx, rr = w / nx;
                const int py = rr % TYH, c = rr / TYH;
                const int gy = y0 - 1 + py;
                const bool in = (unsigned)gy < (unsigned)ny && py <= TY + 1;
                Pt[(c * TYH + py) * LX + x] = in ? __ldg(&Pc[c * S.ncell + ((long)z * ny + gy) * nx + x]) : 0.f;
            }
        }
    }
    __syncthreads();
    // bit r: row r of the block is a bulk row (rows r - 1, r, r + 1 = tile rows r .. r + 2 all good)
    const unsigned badrows = s_bad, badrows2 = s_bad2;
    const unsigned bulk_rows = (m0x4 != 0u && MODE != MODE_XFWD)
                                   ? ~(badrows | (badrows >> 1) | (badrows >> 2)) & ((1u << TY) - 1u) : 0u;
    // rows whose cells see only material m0 or the outside of the grid (a superset of the bulk rows)
    const unsigned box_rows = (m0x4 != 0u && MODE != MODE_XFWD)
                                  ? ~(badrows2 | (badrows2 >> 1) | (badrows2 >> 2)) & ((1u << TY) - 1u) : 0u;
    const int m0 = (int)(m0x4 & 0xffu);
    const unsigned other_rows = ~bulk_rows & ((1u << TY) - 1u);
    if (tid < TY) {
        const unsigned below = (1u << tid) - 1u;
        if ((bulk_rows >> tid) & 1u) s_rowidx[0][__popc(bulk_rows & below)] = (unsigned char)tid;
        else s_rowidx[1][__popc(other_rows & below)] = (unsigned char)tid;
    }
    __syncthreads();
    // ---- cells
    const TileView<LX, TYH, SHORT> V{Pt, Pc, S.ncell, {((long)(z - 1) * ny + y0 - 1) * nx, ((long)(z + 1) * ny + y0 - 1) * nx},
                                     Mt, nx};
    // The sim's scalars and material m0's coefficients in registers: the cell loops store to global
    // memory, after which every field of the descriptor (itself in global memory) would be reloaded.
    const long ncell = S.ncell;
    const unsigned terms = S.terms;
    const bool cross = S.has_cross != 0;
    const float dtc = S.dt, pmax = S.pmax, oscale = S.out_scale;
    float *const hbuf = S.hbuf;
    float *const outp = S.out;
    float land0[8], gd[3], go[3], wxy = 0.f, wxz = 0.f, wyz = 0.f;
    const float inv2d[3] = {S.inv_2d[0], S.inv_2d[1], S.inv_2d[2]};
    const float c10 = s_coef[m0 * NCOEF + 10], c11 = s_coef[m0 * NCOEF + 11];
    {
        const float *c0 = s_coef + m0 * NCOEF;
#pragma unroll
        for (int i = 0; i < 8; ++i) land0[i] = c0[i];
        const float i2[3] = {S.inv_d2[0], S.inv_d2[1], S.inv_d2[2]};
#pragma unroll
        for (int d = 0; d < 3; ++d) { gd[d] = c0[8] * i2[d]; go[d] = c0[9] * i2[d]; }
        if (cross) {
            const float C = c0[10] + c0[11];
            wxy = C * S.inv_2d[0] * S.inv_2d[1];
            wxz = C * S.inv_2d[0] * S.inv_2d[2];
            wyz = C * S.inv_2d[1] * S.inv_2d[2];
        }
    }
    const float *const zlo = Pc + V.row0[0];   // plane z - 1, tile row 0, x 0 (component 0)
    const float *const zhi = Pc + V.row0[1];   // plane z + 1
    float lmax = 0.f;
    bool bad = false;
    // energy sums of this thread's few cells in float32 (their densities are float32), widened to
    // float64 once for the block and grid sums: one conversion per thread and term instead of a
    // float64 add per cell, which this part's FP64 rate would make the energy pass's bottleneck
    float e_land = 0.f, e_grad = 0.f, e_elec = 0.f, e_ext = 0.f;
    // Gradient field of a bulk cell of material m0 (all 18 neighbours inside the grid and of m0):
    // the discrete Eq. 4 reduces to G (P(+) + P(-) - 2P) / dx^2 per face pair plus
    // (G12 + G44 - G'44) times the four-corner mixed differences d_e d_f P_f (tgrad_field's bulk form).
    auto bulk_grad = [&](const int py, const int x, const float *p, float *h) {
        constexpr int TS = TYH * LX;                  // component stride of the shared tile
        const float *c = Pt + py * LX + x;            // centre plane, component 0
        const float *lo = zlo + py * nx + x, *hi = zhi + py * nx + x;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const float lx = c[i * TS - 1] + c[i * TS + 1] - 2.f * p[i];
            const float ly = c[i * TS - LX] + c[i * TS + LX] - 2.f * p[i];
            const float lz = __ldg(lo + i * ncell) + __ldg(hi + i * ncell) - 2.f * p[i];
            h[i] = fmaf(i == 0 ? gd[0] : go[0], lx, fmaf(i == 1 ? gd[1] : go[1], ly, fmaf(i == 2 ? gd[2] : go[2], lz, h[i])));
        }
        if (cross) {
            // (x+,y+) - (x+,y-) - (x-,y+) + (x-,y-) and the xz / yz analogues
            auto cxy = [&](int f) {
                const float *q = c + f * TS;
                return q[LX + 1] - q[-LX + 1] - q[LX - 1] + q[-LX - 1];
            };
            auto cxz = [&](int f) {
                const float *a = hi + f * ncell, *b = lo + f * ncell;
                return (__ldg(a + 1) - __ldg(b + 1)) - (__ldg(a - 1) - __ldg(b - 1));
            };
            auto cyz = [&](int f) {
                const float *a = hi + f * ncell, *b = lo + f * ncell;
                return (__ldg(a + nx) - __ldg(b + nx)) - (__ldg(a - nx) - __ldg(b - nx));
            };
            h[0] = fmaf(wxy, cxy(1), fmaf(wxz, cxz(2), h[0]));
            h[1] = fmaf(wxy, cxy(0), fmaf(wyz, cyz(2), h[1]));
            h[2] = fmaf(wxz, cxz(0), fmaf(wyz, cyz(1), h[2]));
        }
    };
    // Gradient field of a cell whose neighbours inside the grid are all of material m0 while some
    // lie outside it (grid faces, edges and corners of a one-material region): the ghost rules of
    // the discrete Eq. 4 (no face term to the outside; mirror ghosts in the central differences; odd
    // ghosts for the cross fluxes) with in-grid flags taken from the coordinates instead of the
    // material tile, and m0's coefficients in registers.  The operations and their order are those
    // of tgrad_field's general form, so both give the same result bit for bit.
    auto box_grad = [&](const int py, const int x, const float *pa, float *h) {
        const int gy = y0 - 1 + py;
        const bool fin[3][2] = {{x > 0, x < nx - 1}, {gy > 0, gy < ny - 1}, {z > 0, z < nz - 1}};
        // P_f at offset (dz, dy, dx) from the cell; an offset outside the grid reads the cell itself
        auto P = [&](int f, int dz, int dy, int dx) -> float {
            if (dx < 0 && !fin[0][0]) dx = 0;
            if (dx > 0 && !fin[0][1]) dx = 0;
            if (dy < 0 && !fin[1][0]) dy = 0;
            if (dy > 0 && !fin[1][1]) dy = 0;
            if (dz < 0 && !fin[2][0]) dz = 0;
            if (dz > 0 && !fin[2][1]) dz = 0;
            return V.p(f, 1 + dz, py + dy, x + dx);
        };
        auto in = [&](int dz, int dy, int dx) {
            return (dx >= 0 || fin[0][0]) && (dx <= 0 || fin[0][1]) && (dy >= 0 || fin[1][0]) &&
                   (dy <= 0 || fin[1][1]) && (dz >= 0 || fin[2][0]) && (dz <= 0 || fin[2][1]);
        };
        auto off = [](int d, int s, int &dz, int &dy, int &dx) {
            if (d == 0) dx += s; else if (d == 1) dy += s; else dz += s;
        };
        // D_a P_f at offset q (mirror ghosts)
        auto tc = [&](int qz, int qy, int qx, int a, int f) {
            const float q0 = P(f, qz, qy, qx);
            int az = qz, ay = qy, ax = qx, bz = qz, by = qy, bx = qx;
            off(a, 1, az, ay, ax);
            off(a, -1, bz, by, bx);
            const float qp = in(az, ay, ax) ? P(f, az, ay, ax) : q0;
            const float qm = in(bz, by, bx) ? P(f, bz, by, bx) : q0;
            return (qp - qm) * inv2d[a];
        };
        auto fl = [&](int qz, int qy, int qx, int d, float &Sd, float *T) {
            float s = 0.f;
#pragma unroll
            for (int j = 0; j < 3; ++j)
                if (j != d) s += tc(qz, qy, qx, j, j);
            Sd = c10 * s;
#pragma unroll
            for (int i = 0; i < 3; ++i) T[i] = (i != d) ? c11 * tc(qz, qy, qx, i, d) : 0.f;
        };
#pragma unroll
        for (int d = 0; d < 3; ++d) {
#pragma unroll
            for (int s = -1; s <= 1; s += 2) {
                int dz = 0, dy = 0, dx = 0;
                off(d, s, dz, dy, dx);
                if (!in(dz, dy, dx)) continue;
#pragma unroll
                for (int i = 0; i < 3; ++i) h[i] = fmaf(i == d ? gd[d] : go[d], P(i, dz, dy, dx) - pa[i], h[i]);
            }
        }
        if (!cross) return;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            float Sa, Ta[3], Sp, Tp[3], Sm, Tm[3];
            fl(0, 0, 0, d, Sa, Ta);
            int az = 0, ay = 0, ax = 0, bz = 0, by = 0, bx = 0;
            off(d, 1, az, ay, ax);
            off(d, -1, bz, by, bx);
            if (in(az, ay, ax)) fl(az, ay, ax, d, Sp, Tp);
            else { Sp = -Sa; Tp[0] = -Ta[0]; Tp[1] = -Ta[1]; Tp[2] = -Ta[2]; }
            if (in(bz, by, bx)) fl(bz, by, bx, d, Sm, Tm);
            else { Sm = -Sa; Tm[0] = -Ta[0]; Tm[1] = -Ta[1]; Tm[2] = -Ta[2]; }
            const float w = inv2d[d];
            h[d] = fmaf(Sp - Sm, w, h[d]);
#pragma unroll
            for (int i = 0; i < 3; ++i)
                if (i != d) h[i] = fmaf(Tp[i] - Tm[i], w, h[i]);
        }
    };
    // Gradient energy density of a bulk cell of material m0: tgrad_energy's faces towards +x, +y, +z
    // and cross terms, whose ghost rules never apply here, with m0's coefficients in registers
    // (the same operations in the same order, so both give the same result bit for bit).
    auto bulk_genergy = [&](const int py, const int x, const float *pa) {
        constexpr int TS = TYH * LX;
        const float *c = Pt + py * LX + x;
        const float *hi = zhi + py * nx + x, *lo = zlo + py * nx + x;
        float e = 0.f;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const float g = 0.5f * ((i == d) ? gd[d] + gd[d] : go[d] + go[d]);
                const float nb = d == 0 ? c[i * TS + 1] : (d == 1 ? c[i * TS + LX] : __ldg(hi + i * ncell));
                const float df = nb - pa[i];
                e = fmaf(0.5f * g * df, df, e);
            }
        }
        if (cross) {
            float D[3][3];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                D[i][0] = (c[i * TS + 1] - c[i * TS - 1]) * inv2d[0];
                D[i][1] = (c[i * TS + LX] - c[i * TS - LX]) * inv2d[1];
                D[i][2] = (__ldg(hi + i * ncell) - __ldg(lo + i * ncell)) * inv2d[2];
            }
            e += c10 * (D[0][0] * D[1][1] + D[1][1] * D[2][2] + D[2][2] * D[0][0]) +
                 c11 * (D[0][1] * D[1][0] + D[1][2] * D[2][1] + D[0][2] * D[2][0]);
        }
        return e;
    };
    // the rest of a cell once its Landau and gradient fields are in h: E_el, E_ext, then the mode's
    // output (field, dP/dt) or update
    auto finish = [&](const int r, const int x, const float *p, float *h) {
        const long id = ((long)z * ny + y0 + r) * nx + x;
        if (elec) {
#pragma unroll
            for (int c = 0; c < 3; ++c) h[c] += Eb[(c * TYmax + r) * LX + x];
        }
        if (terms & TERM_EXT) {
#pragma unroll
            for (int c = 0; c < 3; ++c) h[c] += eext[c];
        }
        if (MODE == MODE_FIELD) {
#pragma unroll
            for (int c = 0; c < 3; ++c) outp[c * ncell + id] = h[c] * oscale;
            return;
        }
        if (MODE == MODE_DERIV) {   // dP/dt of Eq. 1 (L = 1, normalized) for a multi-stage integrator
#pragma unroll
            for (int c = 0; c < 3; ++c) hbuf[c * ncell + id] = h[c];
            return;
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float pn, p0 = p[c];
            if (MODE == MODE_HEUN2) {
                p0 = Pn[c * ncell + id];
                pn = fmaf(0.5f * dtc, hbuf[c * ncell + id] + h[c], p0);
            } else {
                pn = fmaf(dtc, h[c], p0);
                if (MODE == MODE_HEUN1) hbuf[c * ncell + id] = h[c];
            }
            if (MODE != MODE_HEUN1) lmax = fmaxf(lmax, fabsf(pn - p0));
            bad |= !(fabsf(pn) <= pmax);
            Pn[c * ncell + id] = pn;
            Eb[(c * TYmax + r) * LX + x] = pn;      // the cell's own slot: E read above, new P kept
        }
    };
    // one cell (r, x); BULK: known bulk cell of material m0 (no vacuum, ghost or interface rule)
    auto cell = [&](const int r, const int x, const auto kind_tag) {
        constexpr int KIND = decltype(kind_tag)::value;   // 0 general, 1 bulk, 2 box boundary
        constexpr bool BULK = KIND == 1, KNOWN = KIND != 0;
        const int py = r + 1;
        const long id = ((long)z * ny + y0 + r) * nx + x;
        const int m = KNOWN ? m0 : V.m(1, py, x);
        if (!KNOWN && m == 0) {
            if (mode_updates(MODE)) {
#pragma unroll
                for (int c = 0; c < 3; ++c) { Pn[c * ncell + id] = 0.f; Eb[(c * TYmax + r) * LX + x] = 0.f; }
            } else if (MODE == MODE_FIELD) {
#pragma unroll
                for (int c = 0; c < 3; ++c) outp[c * ncell + id] = 0.f;
            } else if (MODE == MODE_DERIV) {
#pragma unroll
                for (int c = 0; c < 3; ++c) hbuf[c * ncell + id] = 0.f;
            }
            return;
        }
        float p[3], h[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int c = 0; c < 3; ++c) p[c] = Pt[(c * TYH + py) * LX + x];
        const float *cm = s_coef + m * NCOEF;
        if (MODE == MODE_ENERGY) {
            if (terms & TERM_LANDAU) {
                const float x2 = p[0] * p[0], y2 = p[1] * p[1], z2 = p[2] * p[2];
                const float f = cm[0] * x2 + cm[1] * y2 + cm[2] * z2 + cm[3] * (x2 * x2 + y2 * y2 + z2 * z2) +
                                cm[4] * (x2 * y2 + y2 * z2 + z2 * x2) +
                                cm[5] * (x2 * x2 * x2 + y2 * y2 * y2 + z2 * z2 * z2) +
                                cm[6] * (x2 * x2 * (y2 + z2) + y2 * y2 * (x2 + z2) + z2 * z2 * (x2 + y2)) +
                                cm[7] * x2 * y2 * z2;
                e_land += f;
            }
            if (terms & TERM_GRAD) {
                if constexpr (BULK) e_grad += bulk_genergy(py, x, p);
                else e_grad += tgrad_energy(V, S, s_coef, py, x, m, p);
            }
            float el = 0.f, ex = 0.f;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                if (elec) el = fmaf(-0.5f * Eb[(c * TYmax + r) * LX + x], p[c], el);
                if (terms & TERM_EXT) ex = fmaf(-eext[c], p[c], ex);
            }
            e_elec += el;
            e_ext += ex;
            return;
        }
        if (terms & TERM_LANDAU) {
            if constexpr (KNOWN) landau_field(p, land0, h);
            else landau_field(p, cm, h);
        }
        if (terms & TERM_GRAD) {
            if constexpr (BULK) bulk_grad(py, x, p, h);
            else if constexpr (KIND == 2) box_grad(py, x, p, h);
            else tgrad_field(V, S, s_coef, py, x, m, p, h, false);
        }
        finish(r, x, p, h);
    };
    if (MODE != MODE_XFWD) {
        // bulk pass: cells 1 .. nx - 2 of the bulk rows, warp-uniform fast path
        const int nb = __popc(bulk_rows);
        for (int w = tid; w < nb * (nx - 2); w += nthr) {
            const int j = w / (nx - 2), x = 1 + w - j * (nx - 2);
            cell((int)s_rowidx[0][j], x, std::integral_constant<int, 1>{});
        }
        // general pass: every cell of the other rows, then the two end cells of each bulk row
        const int nrest = (TY - nb) * nx;
        for (int w = tid; w < nrest + 2 * nb; w += nthr) {
            if (w < nrest) {
                const int j = w / nx, x = w - j * nx;
                const int r = (int)s_rowidx[1][j];
                if ((box_rows >> r) & 1u) cell(r, x, std::integral_constant<int, 2>{});
                else cell(r, x, std::integral_constant<int, 0>{});
            } else {
                const int k = w - nrest;
                cell((int)s_rowidx[0][k >> 1], (k & 1) ? nx - 1 : 0, std::integral_constant<int, 2>{});
            }
        }
    }
    if (MODE == MODE_ENERGY) {
        double v;
        v = block_sum((double)e_land, s_red); if (tid == 0) atomicAdd(&S.energy[0], v);
        v = block_sum((double)e_grad, s_red); if (tid == 0) atomicAdd(&S.energy[1], v);
        v = block_sum((double)e_elec, s_red); if (tid == 0) atomicAdd(&S.energy[2], v);
        v = block_sum((double)e_ext, s_red); if (tid == 0) atomicAdd(&S.energy[3], v);
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
        const float *src = (MODE == MODE_XFWD) ? Pt + (lc * TYH + lr + 1) * LX : Eb + (lc * TYmax + lr) * LX;
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
