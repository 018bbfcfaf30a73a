// Device side of libtdgl: one explicit TDGL step (Eq. 1) as four kernels, plus the FP64 build
// of the cell-interaction tensor spectrum and small helpers.
//
//   k_rows<STEP>  for each x-row: C2R x-inverse of the field spectrum -> E_el row; Landau field
//                 (Eq. 3), gradient field (Eq. 4, discrete), E_ext (Eq. 7); forward Euler update
//                 of P; R2C x-forward of the new P row (zero-padded to Mx).
//   k_yfwd        y forward FFT (zero-padded ny -> My) of the x-spectrum.
//   k_zconv       z forward FFT (nz -> Mz), per-k 3x3 tensor multiply (Eqs. 5-6 as a
//                 convolution), z inverse FFT keeping the first nz outputs.
//   k_yinv        y inverse FFT keeping the first ny outputs.
//
// Normalized float32 inside (Table 2): P* = P/P0, t* = alpha_ref L t, E* = E/(alpha_ref P0),
// lengths in units of the smallest cell edge.  Every kernel takes a table of sim descriptors
// and a table of work items, so one launch covers a single sim or a batch of uneven sims.
#pragma once
#include "philox.cuh"
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fft.cuh"

namespace tdgl {

enum { TERM_LANDAU = 1, TERM_GRAD = 2, TERM_ELEC = 4, TERM_EXT = 8 };
enum { NCOEF = 12 };  // a1x a1y a1z a11 a12 a111 a112 a123 G11 G44s G12 Gd (normalized)
enum { MAXMAT = 16 };
enum { NTHREADS = 256 };

struct SimDev {
    int nx, ny, nz;
    long ncell;
    int hx, Kx, kxp;          // x: complex length Mx/2, kept planes Mx/2+1, row pitch (complex)
    int My, Mz;               // padded y and z lengths
    int kyh, kzh;             // My/2+1, Mz/2+1 (rows of the reduced tensor spectrum)
    Plan px, py, pz;          // complex FFT plans (x: length hx)
    int twr;                  // offset of W_Mx^k, k in [0, hx], in tw
    const float2 *tw;         // twiddle tables
    float *P[2];              // normalized P, double buffer, [3][ncell]
    const uint8_t *mat;       // [ncell]
    float2 *X;                // [3][nz][ny][kxp]  x-spectrum (P-hat or E-hat)
    float2 *Y;                // [3][nz][My][kxp]  y-padded spectrum
    const float2 *Nhat;       // [3][kzh][kyh][kxp] reduced real tensor spectrum, (xx,yy) (zz,xy) (xz,yz)
    const float *coef;        // [MAXMAT][NCOEF]
    float inv_d2[3];          // 1/dx*^2
    float inv_2d[3];          // 1/(2 dx*)
    float dt;                 // alpha_ref L dt
    float eext[3];            // E_ext / (alpha_ref P0), static part
    float eac[3];             // amplitude of the sinusoidal part, normalized like eext
    double ac_ph0, ac_dph;    // its phase at the first step of the call and per step
    float escale;             // -1/(eps0 epsB alpha_ref) / (Mx My Mz)
    float pmax;               // divergence bound on |P*_i|
    unsigned terms;
    int has_cross;
    unsigned *maxdp;          // float bits of max |dP*| of the step
    int *flag;                // bit 0: divergence; bit 1: a bounded pipeline wait timed out
    double *energy;           // [4] land grad elec ext, normalized (times alpha_ref P0^2 V -> J)
    float *out;               // field readback [3][ncell]
    float *hbuf;              // Heun: field of the predictor's starting point [3][ncell]
    float out_scale;          // alpha_ref P0
    int skip;                 // nonzero: every step kernel returns at once for this sim (a batch
                              // member the device relaxation loop has retired)
    int has_ymap;             // ymap below is valid (the z pass then loads its lines with TMA)
    // Y viewed as float32 (2 kxp, My, nz, 3), box (2 x lines per block, 1, nz, 1): the z lines of
    // one ky and one group of kx, one component per copy
    alignas(64) CUtensorMap ymap;
    int has_nmap;             // nmap below is valid (staged z-pass variant)
    // Nhat viewed as float32 (2 kxp, kyh, kzh, 3), box (2 x lines per block, 1, kzh, 1): the rows
    // of one reduced ky for one group of kx, one component pair per copy
    alignas(64) CUtensorMap nmap;
};

// State of the device-side relaxation loop (the relaxation to equilibrium of Sec. 2): steps done,
// the step cap, the tolerance on max |dP*| of a step and the steps per loop body.
struct RelaxState {
    long done, max_steps;
    double tol;
    int k;
};

// work item: x = sim index, y/z/w kernel specific
//   rows kernels: y = z, z = y0, w = row count
//   y kernels:    y = c*nz + z, z = kx0, w = kx count
//   z kernel:     y = ky, z = kx0, w = kx count

// STEP: forward Euler.  HEUN1 / HEUN2: predictor and corrector of Heun's method (Sec. 3):
//   HEUN1  P~ = P + dt h(P), keeps h(P) in S.hbuf, writes P~ to the other buffer;
//   HEUN2  P <- P + dt/2 (h(P) + h(P~)) in place, with the field evaluated on P~.
// DERIV: the total field (= dP/dt of Eq. 1 with L = 1, normalized) of the state in P[parity],
// written to hbuf; the stages of the Runge-Kutta-Fehlberg and Adams integrators are built from it
enum { MODE_STEP = 0, MODE_FIELD = 1, MODE_ENERGY = 2, MODE_XFWD = 3, MODE_HEUN1 = 4, MODE_HEUN2 = 5, MODE_DERIV = 6 };
__host__ __device__ constexpr bool mode_updates(int m) { return m == MODE_STEP || m == MODE_HEUN1 || m == MODE_HEUN2; }

__device__ __forceinline__ int row_ld(const SimDev &S) { return S.hx + 2; }

// ---- Landau field, Eq. 3 (h = -df/dP) -----------------------------------------------------
__device__ __forceinline__ void landau_field(const float *p, const float *c, float *h) {
    const float x2 = p[0] * p[0], y2 = p[1] * p[1], z2 = p[2] * p[2];
    const float sq[3] = {x2, y2, z2};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float pi2 = sq[i], pj2 = sq[(i + 1) % 3], pk2 = sq[(i + 2) % 3];
        const float o2 = pj2 + pk2;
        float d = 2.f * c[i];                       // 2 a1_i
        d = fmaf(4.f * c[3], pi2, d);               // 4 a11 P_i^2
        d = fmaf(2.f * c[4], o2, d);                // 2 a12 (P_j^2 + P_k^2)
        d = fmaf(6.f * c[5], pi2 * pi2, d);         // 6 a111 P_i^4
        d = fmaf(c[6], fmaf(4.f * pi2, o2, 2.f * (pj2 * pj2 + pk2 * pk2)), d);  // a112 terms
        d = fmaf(2.f * c[7], pj2 * pk2, d);         // 2 a123 P_j^2 P_k^2
        h[i] -= d * p[i];
    }
}

// Landau energy density in float64 (normalized)
__device__ __forceinline__ double landau_energy(const float *pf, const float *c) {
    const double x2 = (double)pf[0] * pf[0], y2 = (double)pf[1] * pf[1], z2 = (double)pf[2] * pf[2];
    return (double)c[0] * x2 + (double)c[1] * y2 + (double)c[2] * z2
         + (double)c[3] * (x2 * x2 + y2 * y2 + z2 * z2)
         + (double)c[4] * (x2 * y2 + y2 * z2 + z2 * x2)
         + (double)c[5] * (x2 * x2 * x2 + y2 * y2 * y2 + z2 * z2 * z2)
         + (double)c[6] * (x2 * x2 * (y2 + z2) + y2 * y2 * (x2 + z2) + z2 * z2 * (x2 + y2))
         + (double)c[7] * x2 * y2 * z2;
}

// applied field of Eq. 7 at step istep of the call: static part plus A sin(phase)
__device__ __forceinline__ void ext_field(const SimDev &S, int istep, float *e) {
    float s = 0.f;
    if (S.eac[0] != 0.f || S.eac[1] != 0.f || S.eac[2] != 0.f) s = (float)sin(S.ac_ph0 + istep * S.ac_dph);
#pragma unroll
    for (int c = 0; c < 3; ++c) e[c] = fmaf(S.eac[c], s, S.eext[c]);
}

// ---- neighbourhood access with the free-surface rules of the discrete Eq. 4 ----------------
struct Cell {
    int x, y, z;
};

__device__ __forceinline__ bool inside(const SimDev &S, int x, int y, int z) {
    return (unsigned)x < (unsigned)S.nx && (unsigned)y < (unsigned)S.ny && (unsigned)z < (unsigned)S.nz;
}
__device__ __forceinline__ long cidx(const SimDev &S, int x, int y, int z) {
    return ((long)z * S.ny + y) * S.nx + x;
}
__device__ __forceinline__ int matat(const SimDev &S, int x, int y, int z) {
    return inside(S, x, y, z) ? (int)__ldg(&S.mat[cidx(S, x, y, z)]) : 0;
}
__device__ __forceinline__ void step3(int d, int s, int &x, int &y, int &z) {
    if (d == 0) x += s; else if (d == 1) y += s; else z += s;
}

// central difference D_d P_f at a material cell with mirror ghosts
__device__ __forceinline__ float central(const SimDev &S, const float *Pc, int x, int y, int z, int d, int f) {
    const long base = (long)f * S.ncell;
    const float q0 = __ldg(&Pc[base + cidx(S, x, y, z)]);
    int xp = x, yp = y, zp = z, xm = x, ym = y, zm = z;
    step3(d, 1, xp, yp, zp);
    step3(d, -1, xm, ym, zm);
    const float qp = matat(S, xp, yp, zp) ? __ldg(&Pc[base + cidx(S, xp, yp, zp)]) : q0;
    const float qm = matat(S, xm, ym, zm) ? __ldg(&Pc[base + cidx(S, xm, ym, zm)]) : q0;
    return (qp - qm) * S.inv_2d[d];
}

// Fluxes of the cross terms at material cell (x,y,z) attached to direction d:
//   Sd      = G12 * sum_{j != d} D_j P_j          (multiplies D_d P_d)
//   T[i]    = Gd  * D_i P_d for i != d            (multiplies D_d P_i)
__device__ __forceinline__ void cross_fluxes(const SimDev &S, const float *Pc, const float *coef,
                                             int x, int y, int z, int m, int d, float &Sd, float *T) {
    const float *c = coef + m * NCOEF;
    const float G12 = c[10], Gd = c[11];
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 3; ++j)
        if (j != d) s += central(S, Pc, x, y, z, j, j);
    Sd = G12 * s;
#pragma unroll
    for (int i = 0; i < 3; ++i) T[i] = (i != d) ? Gd * central(S, Pc, x, y, z, i, d) : 0.f;
}

// gradient field (Eq. 4, discrete form: faces + cross terms) at material cell a
__device__ __forceinline__ void gradient_field(const SimDev &S, const float *Pc, const float *coef,
                                               int x, int y, int z, int ma, const float *pa, float *h) {
    const float *ca = coef + ma * NCOEF;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
#pragma unroll
        for (int s = -1; s <= 1; s += 2) {
            int xn = x, yn = y, zn = z;
            step3(d, s, xn, yn, zn);
            const int mb = matat(S, xn, yn, zn);
            if (!mb) continue;
            const float *cb = coef + mb * NCOEF;
            const long nb = cidx(S, xn, yn, zn);
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const float ga = (i == d) ? ca[8] : ca[9];
                const float gb = (i == d) ? cb[8] : cb[9];
                const float g = 0.5f * (ga + gb) * S.inv_d2[d];
                h[i] = fmaf(g, __ldg(&Pc[(long)i * S.ncell + nb]) - pa[i], h[i]);
            }
        }
    }
    if (!S.has_cross) return;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        float Sa, Ta[3];
        cross_fluxes(S, Pc, coef, x, y, z, ma, d, Sa, Ta);
        float Sp, Tp[3], Sm, Tm[3];
        int xp = x, yp = y, zp = z, xm = x, ym = y, zm = z;
        step3(d, 1, xp, yp, zp);
        step3(d, -1, xm, ym, zm);
        const int mp = matat(S, xp, yp, zp), mm = matat(S, xm, ym, zm);
        if (mp) cross_fluxes(S, Pc, coef, xp, yp, zp, mp, d, Sp, Tp);
        else { Sp = -Sa; Tp[0] = -Ta[0]; Tp[1] = -Ta[1]; Tp[2] = -Ta[2]; }
        if (mm) cross_fluxes(S, Pc, coef, xm, ym, zm, mm, d, Sm, Tm);
        else { Sm = -Sa; Tm[0] = -Ta[0]; Tm[1] = -Ta[1]; Tm[2] = -Ta[2]; }
        const float w = S.inv_2d[d];
        h[d] = fmaf(Sp - Sm, w, h[d]);
#pragma unroll
        for (int i = 0; i < 3; ++i)
            if (i != d) h[i] = fmaf(Tp[i] - Tm[i], w, h[i]);
    }
}

// gradient energy density at material cell a: faces towards +x, +y, +z and the cross terms
__device__ __forceinline__ double gradient_energy(const SimDev &S, const float *Pc, const float *coef,
                                                  int x, int y, int z, int ma, const float *pa) {
    const float *ca = coef + ma * NCOEF;
    double e = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        int xn = x, yn = y, zn = z;
        step3(d, 1, xn, yn, zn);
        const int mb = matat(S, xn, yn, zn);
        if (!mb) continue;
        const float *cb = coef + mb * NCOEF;
        const long nb = cidx(S, xn, yn, zn);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const double g = 0.5 * ((i == d) ? (double)ca[8] + cb[8] : (double)ca[9] + cb[9]) * S.inv_d2[d];
            const double df = (double)__ldg(&Pc[(long)i * S.ncell + nb]) - pa[i];
            e += 0.5 * g * df * df;
        }
    }
    if (S.has_cross) {
        double D[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int d = 0; d < 3; ++d) D[i][d] = central(S, Pc, x, y, z, d, i);
        e += (double)ca[10] * (D[0][0] * D[1][1] + D[1][1] * D[2][2] + D[2][2] * D[0][0])
           + (double)ca[11] * (D[0][1] * D[1][0] + D[1][2] * D[2][1] + D[0][2] * D[2][0]);
    }
    return e;
}

__device__ __forceinline__ double block_sum(double v, double *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x < 32) {
        r = (lane < (int)(blockDim.x >> 5)) ? red[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    }
    return r;
}

// ---- the row kernel ---------------------------------------------------------------------------
// smem: bufA, bufB each [3][cnt][ld] float2 with ld = hx + 2; coefficient table; reduction.
template <int MODE>
__global__ void __launch_bounds__(NTHREADS) k_rows(const SimDev *__restrict__ sims, const int4 *__restrict__ items,
                                                   int istep) {
    extern __shared__ float4 smem4[];
    __shared__ float s_coef[MAXMAT * NCOEF];
    __shared__ double s_red[NTHREADS / 32];
    __shared__ float s_max;
    const int4 it = items[blockIdx.x];
    const SimDev &S = sims[it.x];
    if (S.skip) return;   // a batch member that has left the relaxation
    const int z = it.y, y0 = it.z, cnt = it.w;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int ld = row_ld(S);
    const int nl = 3 * cnt;
    float2 *bufA = reinterpret_cast<float2 *>(smem4);
    float2 *bufB = bufA + nl * ld;
    for (int i = tid; i < MAXMAT * NCOEF; i += nthr) s_coef[i] = S.coef[i];
    if (tid == 0) s_max = 0.f;
    const int parity = istep & 1;      // istep: step index within the call
    // HEUN2 evaluates the field on the predictor (other buffer) and updates P in place
    const float *Pc = (MODE == MODE_HEUN2) ? S.P[parity ^ 1] : S.P[parity];
    float *Pn = (MODE == MODE_HEUN2) ? S.P[parity] : S.P[parity ^ 1];
    const bool elec = (S.terms & TERM_ELEC) != 0;
    const int nx = S.nx, hx = S.hx;
    float eext[3];
    ext_field(S, istep, eext);
    const float2 *twr = S.tw + S.twr;

    float *Erow = nullptr;   // float view: line l holds E*_c of row r at [l*2*ld + x]
    float2 *Qbuf = bufA;     // new-P rows (float view) for the forward transform
    float2 *Wbuf = bufB;
    if (MODE != MODE_XFWD && elec) {
        // load the field spectrum rows X[c][z][y0+r][k], k <= hx
        for (int w = tid; w < nl * S.Kx; w += nthr) {
            const int l = w / S.Kx, k = w - l * S.Kx;
            const int c = l / cnt, r = l - c * cnt;
            bufA[l * ld + k] = S.X[(((long)c * S.nz + z) * S.ny + y0 + r) * S.kxp + k];
        }
        __syncthreads();
        // Hermitian half-spectrum -> packed complex spectrum of length hx
        for (int w = tid; w < nl * hx; w += nthr) {
            const int l = w / hx, k = w - l * hx;
            const float2 a = bufA[l * ld + k];
            const float2 b = cconj(bufA[l * ld + hx - k]);
            float2 t = twr[k];
            t.y = -t.y;   // W^{-k}
            const float2 d = cmul(csub(a, b), t);
            bufB[l * ld + k] = make_float2(a.x + b.x - d.y, a.y + b.y + d.x);   // (a+b) + i d
        }
        __syncthreads();
        float2 *res = fft_lines<true>(bufB, bufA, S.px, nl, ld, S.tw, tid, nthr);
        Erow = reinterpret_cast<float *>(res);
        Qbuf = (res == bufA) ? bufB : bufA;
        Wbuf = res;
    }

    float lmax = 0.f;
    bool bad = false;
    double e_land = 0.0, e_grad = 0.0, e_elec = 0.0, e_ext = 0.0;
    float *Q = reinterpret_cast<float *>(Qbuf);
    __syncthreads();
    if (MODE == MODE_XFWD) {
        for (int w = tid; w < nl * nx; w += nthr) {
            const int l = w / nx, x = w - l * nx;
            const int c = l / cnt, r = l - c * cnt;
            Q[l * 2 * ld + x] = Pc[(long)c * S.ncell + cidx(S, x, y0 + r, z)];
        }
    } else {
        for (int w = tid; w < cnt * nx; w += nthr) {
            const int r = w / nx, x = w - r * nx;
            const int y = y0 + r;
            const long id = cidx(S, x, y, z);
            const int m = __ldg(&S.mat[id]);
            if (m == 0) {
                if (mode_updates(MODE)) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) { Pn[c * S.ncell + id] = 0.f; Q[(c * cnt + r) * 2 * ld + x] = 0.f; }
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
            for (int c = 0; c < 3; ++c) p[c] = Pc[c * S.ncell + id];
            const float *cm = s_coef + m * NCOEF;
            if (MODE == MODE_ENERGY) {
                if (S.terms & TERM_LANDAU) e_land += landau_energy(p, cm);
                if (S.terms & TERM_GRAD) e_grad += gradient_energy(S, Pc, s_coef, x, y, z, m, p);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    if (elec) e_elec += -0.5 * (double)Erow[(c * cnt + r) * 2 * ld + x] * p[c];
                    if (S.terms & TERM_EXT) e_ext += -(double)eext[c] * p[c];
                }
                continue;
            }
            if (S.terms & TERM_LANDAU) landau_field(p, cm, h);
            if (S.terms & TERM_GRAD) gradient_field(S, Pc, s_coef, x, y, z, m, p, h);
            if (elec) {
#pragma unroll
                for (int c = 0; c < 3; ++c) h[c] += Erow[(c * cnt + r) * 2 * ld + x];   // scaled in k_zconv
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
                Q[(c * cnt + r) * 2 * ld + x] = pn;
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
        if ((tid & 31) == 0) atomicMax(reinterpret_cast<unsigned *>(&s_max), __float_as_uint(lmax));
        if (bad) atomicOr(S.flag, 1);
    }
    if (!elec) {
        if (mode_updates(MODE)) {
            __syncthreads();
            if (tid == 0) atomicMax(S.maxdp, __float_as_uint(s_max));
        }
        return;
    }
    // zero padding of the new rows, then forward real transform into the x-spectrum
    const int Mx = 2 * hx;
    for (int w = tid; w < nl * (Mx - nx); w += nthr) {
        const int l = w / (Mx - nx), x = nx + (w - l * (Mx - nx));
        Q[l * 2 * ld + x] = 0.f;
    }
    __syncthreads();
    if (mode_updates(MODE) && tid == 0) atomicMax(S.maxdp, __float_as_uint(s_max));
    float2 *res = fft_lines<false>(Qbuf, Wbuf, S.px, nl, ld, S.tw, tid, nthr);
    for (int w = tid; w < nl * S.Kx; w += nthr) {
        const int l = w / S.Kx, k = w - l * S.Kx;
        const int c = l / cnt, r = l - c * cnt;
        const float2 a = res[l * ld + (k == hx ? 0 : k)];
        const float2 b = cconj(res[l * ld + (k == 0 ? 0 : hx - k)]);
        const float2 d = cmul(csub(a, b), twr[k]);                // W^k (Z_k - conj Z_{h-k})
        // X_k = (a + b)/2 - i/2 * d
        S.X[(((long)c * S.nz + z) * S.ny + y0 + r) * S.kxp + k] =
            make_float2(0.5f * (a.x + b.x + d.y), 0.5f * (a.y + b.y - d.x));
    }
}

// ---- y passes ----------------------------------------------------------------------------------
__device__ __forceinline__ int yld(const SimDev &S) { return S.My + 1; }
__device__ __forceinline__ int zld(const SimDev &S) { return S.Mz + 1; }

__global__ void __launch_bounds__(NTHREADS) k_yfwd(const SimDev *__restrict__ sims, const int4 *__restrict__ items) {
    extern __shared__ float4 smem4[];
    const int4 it = items[blockIdx.x];
    const SimDev &S = sims[it.x];
    if (S.skip) return;   // a batch member that has left the relaxation
    const int cz = it.y, kx0 = it.z, cnt = it.w;
    const int tid = threadIdx.x, nthr = blockDim.x, ld = yld(S);
    float2 *A = reinterpret_cast<float2 *>(smem4), *B = A + cnt * ld;
    const float2 *src = S.X + (long)cz * S.ny * S.kxp + kx0;
    for (int w = tid; w < S.My * cnt; w += nthr) {
        const int y = w / cnt, l = w - y * cnt;
        A[l * ld + y] = (y < S.ny) ? src[(long)y * S.kxp + l] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const float2 *res = fft_lines<false>(A, B, S.py, cnt, ld, S.tw, tid, nthr);
    float2 *dst = S.Y + (long)cz * S.My * S.kxp + kx0;
    for (int w = tid; w < S.My * cnt; w += nthr) {
        const int y = w / cnt, l = w - y * cnt;
        dst[(long)y * S.kxp + l] = res[l * ld + y];
    }
}

__global__ void __launch_bounds__(NTHREADS) k_yinv(const SimDev *__restrict__ sims, const int4 *__restrict__ items) {
    extern __shared__ float4 smem4[];
    const int4 it = items[blockIdx.x];
    const SimDev &S = sims[it.x];
    if (S.skip) return;   // a batch member that has left the relaxation
    const int cz = it.y, kx0 = it.z, cnt = it.w;
    const int tid = threadIdx.x, nthr = blockDim.x, ld = yld(S);
    float2 *A = reinterpret_cast<float2 *>(smem4), *B = A + cnt * ld;
    const float2 *src = S.Y + (long)cz * S.My * S.kxp + kx0;
    for (int w = tid; w < S.My * cnt; w += nthr) {
        const int y = w / cnt, l = w - y * cnt;
        A[l * ld + y] = src[(long)y * S.kxp + l];
    }
    __syncthreads();
    const float2 *res = fft_lines<true>(A, B, S.py, cnt, ld, S.tw, tid, nthr);
    float2 *dst = S.X + (long)cz * S.ny * S.kxp + kx0;
    for (int w = tid; w < S.ny * cnt; w += nthr) {
        const int y = w / cnt, l = w - y * cnt;
        dst[(long)y * S.kxp + l] = res[l * ld + y];
    }
}

// ---- z pass with the tensor multiply -----------------------------------------------------------
__global__ void __launch_bounds__(NTHREADS) k_zconv(const SimDev *__restrict__ sims, const int4 *__restrict__ items) {
    extern __shared__ float4 smem4[];
    const int4 it = items[blockIdx.x];
    const SimDev &S = sims[it.x];
    if (S.skip) return;   // a batch member that has left the relaxation
    const int ky = it.y, kx0 = it.z, cnt = it.w;
    const int tid = threadIdx.x, nthr = blockDim.x, ld = zld(S);
    const int nl = 3 * cnt;
    float2 *A = reinterpret_cast<float2 *>(smem4), *B = A + nl * ld;
    const long cstride = (long)S.nz * S.My * S.kxp;     // component stride in Y
    const long zstride = (long)S.My * S.kxp;
    const float2 *src = S.Y + (long)ky * S.kxp + kx0;
    for (int w = tid; w < S.Mz * nl; w += nthr) {
        const int zz = w / nl, l = w - zz * nl;
        const int c = l / cnt, q = l - c * cnt;
        A[l * ld + zz] = (zz < S.nz) ? src[c * cstride + (long)zz * zstride + q] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    float2 *res = fft_lines<false>(A, B, S.pz, nl, ld, S.tw, tid, nthr);
    float2 *oth = (res == A) ? B : A;
    // E-hat = escale * N-hat(k) P-hat(k), N-hat from the reduced table with reflection signs
    const int kyr = (ky <= S.My / 2) ? ky : S.My - ky;
    const float sy = (ky <= S.My / 2) ? 1.f : -1.f;
    const long nstride = (long)S.kzh * S.kyh * S.kxp;
    for (int w = tid; w < S.Mz * cnt; w += nthr) {
        const int kz = w / cnt, q = w - kz * cnt;
        const int kzr = (kz <= S.Mz / 2) ? kz : S.Mz - kz;
        const float sz = (kz <= S.Mz / 2) ? 1.f : -1.f;
        const float2 *N = S.Nhat + ((long)kzr * S.kyh + kyr) * S.kxp + kx0 + q;
        const float2 n0 = __ldg(N), n1 = __ldg(N + nstride), n2 = __ldg(N + 2 * nstride);
        const float nxx = n0.x, nyy = n0.y, nzz = n1.x;
        const float nxy = sy * n1.y, nxz = sz * n2.x, nyz = sy * sz * n2.y;
        const float2 px = res[(0 * cnt + q) * ld + kz], py = res[(1 * cnt + q) * ld + kz],
                     pz = res[(2 * cnt + q) * ld + kz];
        float2 ex, ey, ez;
        ex.x = (nxx * px.x + nxy * py.x + nxz * pz.x) * S.escale;
        ex.y = (nxx * px.y + nxy * py.y + nxz * pz.y) * S.escale;
        ey.x = (nxy * px.x + nyy * py.x + nyz * pz.x) * S.escale;
        ey.y = (nxy * px.y + nyy * py.y + nyz * pz.y) * S.escale;
        ez.x = (nxz * px.x + nyz * py.x + nzz * pz.x) * S.escale;
        ez.y = (nxz * px.y + nyz * py.y + nzz * pz.y) * S.escale;
        res[(0 * cnt + q) * ld + kz] = ex;
        res[(1 * cnt + q) * ld + kz] = ey;
        res[(2 * cnt + q) * ld + kz] = ez;
    }
    __syncthreads();
    const float2 *out = fft_lines<true>(res, oth, S.pz, nl, ld, S.tw, tid, nthr);
    float2 *dst = S.Y + (long)ky * S.kxp + kx0;
    for (int w = tid; w < S.nz * nl; w += nthr) {
        const int zz = w / nl, l = w - zz * nl;
        const int c = l / cnt, q = l - c * cnt;
        dst[c * cstride + (long)zz * zstride + q] = out[l * ld + zz];
    }
}

// ---- P copies with normalization ------------------------------------------------------------------
__global__ void k_scale_in(float *__restrict__ dst, const float *__restrict__ src, const uint8_t *__restrict__ mat,
                           long ncell, float s) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < 3 * ncell; i += (long)gridDim.x * blockDim.x)
        dst[i] = mat[i % ncell] ? src[i] * s : 0.f;
}
__global__ void k_scale_out(float *__restrict__ dst, const float *__restrict__ src, long n, float s) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        dst[i] = src[i] * s;
}
// Linear combination of integrator stages on material cells (vacuum stays 0):
//   out = P + sum_j c[j] K[j];  optionally  errmax = max |sum_j d[j] K[j]|  and  dpmax = max |out - P|
// (coefficients already multiplied by the normalized step), maxima as ordered float bits.
struct Combine {
    float *out;
    const float *P;
    const float *K[7];
    float c[7], d[7];
    int nk, nd;
    const uint8_t *mat;
    long ncell;
    unsigned *errmax, *dpmax;
};
__global__ void k_combine(Combine q) {
    float em = 0.f, dm = 0.f;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < 3 * q.ncell; i += (long)gridDim.x * blockDim.x) {
        if (!q.mat[i % q.ncell]) {
            q.out[i] = 0.f;
            continue;
        }
        const float p = q.P[i];
        float a = 0.f, e = 0.f;
        for (int j = 0; j < q.nk; ++j) a = fmaf(q.c[j], q.K[j][i], a);
        for (int j = 0; j < q.nd; ++j) e = fmaf(q.d[j], q.K[j][i], e);
        const float o = p + a;
        q.out[i] = o;
        em = fmaxf(em, fabsf(e));
        dm = fmaxf(dm, fabsf(o - p));
        if (!(fabsf(o) <= 1e3f)) em = dm = __int_as_float(0x7f800000);   // NaN or |P| > 1e3 P0
    }
    for (int o = 16; o > 0; o >>= 1) {
        em = fmaxf(em, __shfl_xor_sync(0xffffffffu, em, o));
        dm = fmaxf(dm, __shfl_xor_sync(0xffffffffu, dm, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (q.errmax) atomicMax(q.errmax, __float_as_uint(em));
        if (q.dpmax) atomicMax(q.dpmax, __float_as_uint(dm));
    }
}
__global__ void k_mask(float *__restrict__ P, const uint8_t *__restrict__ mat, long ncell) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < 3 * ncell; i += (long)gridDim.x * blockDim.x)
        if (!mat[i % ncell]) P[i] = 0.f;
}

__global__ void k_init_random(float *__restrict__ P, const uint8_t *__restrict__ mat, long ncell,
                              uint32_t k0, uint32_t k1, float amp) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < 3 * ncell; i += (long)gridDim.x * blockDim.x) {
        const long cell = i % ncell;
        const uint32_t c = (uint32_t)(i / ncell);
        const uint32_t u = philox_first((uint32_t)cell, c, 0u, 0u, k0, k1);
        const float v = (float)(2.0 * (((double)u + 0.5) * 2.3283064365386963e-10) - 1.0) * amp;
        P[i] = mat[cell] ? v : 0.f;
    }
}

}  // namespace tdgl
