// Shared-memory mixed-radix FFT building blocks for the zero-padded convolution of Eqs. 5-6.
//
// A line of length n = R_1 R_2 ... R_s is transformed by s Stockham (self-sorting) passes.
// Pass p with radix R and L = R_1...R_{p-1} maps butterfly b in [0, n/R):
//     j = b mod L,   a_r = src[b + r n/R] * W_{L R}^{r j}   (r = 0..R-1),
//     A = DFT_R(a),  dst[(b - j) R + j + q L] = A_q           (q = 0..R-1),
// with W_m = exp(-2 pi i / m) (forward) or its conjugate (inverse, unnormalized).
// Twiddles come from one table of W_n^t, t in [0, n), computed on the host in float64.
#pragma once
#include <cuda_runtime.h>

namespace tdgl {

// radix plan of one complex FFT length
struct Plan {
    int n;       // length
    int nrad;    // number of passes
    int rad[8];  // radices, each one of 16, 8, 4, 3, 2
    int tw;      // offset of the W_n^t table in the sim's twiddle array
};

// Complex sums and differences as packed FP32 pairs: one f32x2 instruction instead of two scalar
// ones, with the same IEEE round-to-nearest results.
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
// a * (-i) in the forward direction, a * (+i) in the inverse direction
template <bool INV> __device__ __forceinline__ float2 rot(float2 a) {
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

template <bool INV> __device__ __forceinline__ void dft2(float2 &a0, float2 &a1) {
    float2 t = a0; a0 = cadd(t, a1); a1 = csub(t, a1);
}

template <bool INV> __device__ __forceinline__ void dft3(float2 &a0, float2 &a1, float2 &a2) {
    const float h = 0.86602540378443864676f;   // sqrt(3)/2
    float2 s = cadd(a1, a2), d = csub(a1, a2);
    float2 m = make_float2(a0.x - 0.5f * s.x, a0.y - 0.5f * s.y);
    float2 r = rot<INV>(cscale(d, h));
    a0 = cadd(a0, s); a1 = cadd(m, r); a2 = csub(m, r);
}

template <bool INV> __device__ __forceinline__ void dft4(float2 &a0, float2 &a1, float2 &a2, float2 &a3) {
    float2 t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3), t3 = rot<INV>(csub(a1, a3));
    a0 = cadd(t0, t2); a2 = csub(t0, t2); a1 = cadd(t1, t3); a3 = csub(t1, t3);
}

// twiddle W_16^k (k = 0..7) for the in-register splits of radix 8 and 16
template <bool INV> __device__ __forceinline__ float2 w16(int k) {
    const float c1 = 0.92387953251128675613f, s1 = 0.38268343236508977173f, r2 = 0.70710678118654752440f;
    float2 w;
    switch (k) {
        case 0: w = make_float2(1.f, 0.f); break;
        case 1: w = make_float2(c1, -s1); break;
        case 2: w = make_float2(r2, -r2); break;
        case 3: w = make_float2(s1, -c1); break;
        case 4: w = make_float2(0.f, -1.f); break;
        case 5: w = make_float2(-s1, -c1); break;
        case 6: w = make_float2(-r2, -r2); break;
        default: w = make_float2(-c1, -s1); break;
    }
    if (INV) w.y = -w.y;
    return w;
}

// radix-8 as two radix-4 transforms of the even and odd samples plus one radix-2 layer
template <bool INV> __device__ __forceinline__ void dft8(float2 *a) {
    float2 e0 = a[0], e1 = a[2], e2 = a[4], e3 = a[6];
    float2 o0 = a[1], o1 = a[3], o2 = a[5], o3 = a[7];
    dft4<INV>(e0, e1, e2, e3);
    dft4<INV>(o0, o1, o2, o3);
    o1 = cmul(o1, w16<INV>(2));
    o2 = rot<INV>(o2);
    o3 = cmul(o3, w16<INV>(6));
    a[0] = cadd(e0, o0); a[4] = csub(e0, o0);
    a[1] = cadd(e1, o1); a[5] = csub(e1, o1);
    a[2] = cadd(e2, o2); a[6] = csub(e2, o2);
    a[3] = cadd(e3, o3); a[7] = csub(e3, o3);
}

template <bool INV> __device__ __forceinline__ void dft16(float2 *a) {
    float2 e[8], o[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) { e[k] = a[2 * k]; o[k] = a[2 * k + 1]; }
    dft8<INV>(e);
    dft8<INV>(o);
#pragma unroll
    for (int k = 1; k < 8; ++k) o[k] = (k == 4) ? rot<INV>(o[k]) : cmul(o[k], w16<INV>(k));
#pragma unroll
    for (int k = 0; k < 8; ++k) { a[k] = cadd(e[k], o[k]); a[k + 8] = csub(e[k], o[k]); }
}

template <int R, bool INV> __device__ __forceinline__ void dft(float2 *a);

// x with (a x) mod m = 1 (m > 1, a and m coprime)
__host__ __device__ constexpr int inv_mod(int a, int m) {
    for (int x = 1; x < m; ++x)
        if ((a * x) % m == 1) return x;
    return 1;
}

// Radices 6 and 12 as prime-factor (Good-Thomas) transforms of coprime lengths N1 N2 (2 x 3,
// 3 x 4).  With the input index n = (N2 n1 + N1 n2) mod N and the output index
// k = (N2 q1 k1 + N1 q2 k2) mod N, q1 = N2^-1 mod N1, q2 = N1^-1 mod N2, the length-N DFT
// factors into N2-point DFTs over n2 followed by N1-point DFTs over n1 with no twiddle factors
// between them (W_N^(nk) = W_N1^(n1 k1) W_N2^(n2 k2) for these index maps).
template <int N1, int N2, bool INV> __device__ __forceinline__ void dft_pfa(float2 *a) {
    constexpr int N = N1 * N2, q1 = inv_mod(N2 % N1, N1), q2 = inv_mod(N1 % N2, N2);
    float2 y[N1][N2];
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) {
        float2 b[N2];
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) b[n2] = a[(N2 * n1 + N1 * n2) % N];
        dft<N2, INV>(b);
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) y[n1][k2] = b[k2];
    }
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) {
        float2 c[N1];
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) c[n1] = y[n1][k2];
        dft<N1, INV>(c);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) a[(N2 * q1 * k1 + N1 * q2 * k2) % N] = c[k1];
    }
}

template <int R, bool INV> __device__ __forceinline__ void dft(float2 *a) {
    if constexpr (R == 2) dft2<INV>(a[0], a[1]);
    else if constexpr (R == 3) dft3<INV>(a[0], a[1], a[2]);
    else if constexpr (R == 4) dft4<INV>(a[0], a[1], a[2], a[3]);
    else if constexpr (R == 6) dft_pfa<2, 3, INV>(a);
    else if constexpr (R == 8) dft8<INV>(a);
    else if constexpr (R == 12) dft_pfa<3, 4, INV>(a);
    else {
        static_assert(R == 16, "radices 2, 3, 4, 6, 8, 12, 16");
        dft16<INV>(a);
    }
}

// One Stockham pass of radix R over `lines` lines (stride ld) from src to dst.
template <int R, bool INV>
__device__ __forceinline__ void stockham_pass(const float2 *__restrict__ src, float2 *__restrict__ dst,
                                              int n, int L, int lines, int ld,
                                              const float2 *__restrict__ tw, int tid, int nthr) {
    const int nb = n / R;
    const int tstride = n / (L * R);
    const int total = nb * lines;
    for (int w = tid; w < total; w += nthr) {
        const int line = w / nb;
        const int b = w - line * nb;
        const int j = b % L;
        const float2 *s = src + line * ld;
        float2 *d = dst + line * ld;
        float2 a[R];
#pragma unroll
        for (int r = 0; r < R; ++r) a[r] = s[b + r * nb];
        if (j != 0) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                float2 t = __ldg(&tw[r * j * tstride]);
                if (INV) t.y = -t.y;
                a[r] = cmul(a[r], t);
            }
        }
        dft<R, INV>(a);
        const int base = (b - j) * R + j;
#pragma unroll
        for (int r = 0; r < R; ++r) d[base + r * L] = a[r];
    }
}

// Full transform of `lines` lines held in buffer a (stride ld); b is scratch of the same size.
// Data must be visible to all threads on entry (caller syncs).  Returns the buffer holding
// the result; all threads are synchronized on return.
template <bool INV>
__device__ float2 *fft_lines(float2 *a, float2 *b, const Plan &p, int lines, int ld,
                             const float2 *__restrict__ twbase, int tid, int nthr) {
    const float2 *tw = twbase + p.tw;
    int L = 1;
    for (int s = 0; s < p.nrad; ++s) {
        const int R = p.rad[s];
        switch (R) {
            case 16: stockham_pass<16, INV>(a, b, p.n, L, lines, ld, tw, tid, nthr); break;
            case 8: stockham_pass<8, INV>(a, b, p.n, L, lines, ld, tw, tid, nthr); break;
            case 4: stockham_pass<4, INV>(a, b, p.n, L, lines, ld, tw, tid, nthr); break;
            case 3: stockham_pass<3, INV>(a, b, p.n, L, lines, ld, tw, tid, nthr); break;
            default: stockham_pass<2, INV>(a, b, p.n, L, lines, ld, tw, tid, nthr); break;
        }
        __syncthreads();
        float2 *t = a; a = b; b = t;
        L *= R;
    }
    return a;
}

}  // namespace tdgl
