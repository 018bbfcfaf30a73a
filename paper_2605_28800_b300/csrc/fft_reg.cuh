// Register-resident FFT of compile-time length N for groups of T = N/E threads per line.
//
// A shape S fixes N, the elements per thread E and up to three radices R0 R1 R2 (R0 R1 R2 = N,
// each dividing E).  On entry thread t holds v[m] = x[t + T m] (m < E), which is exactly the
// input of the first Stockham pass (see fft.cuh for the pass definition): butterfly u of thread
// t is b = t + T u and reads elements b + r N/R_1, i.e. registers m = u + r E/R_1.  Between
// passes the outputs go through a shared-memory exchange buffer addressed by a caller functor
// idx(pos) (layout chosen by the caller for conflict-free, coalesced access); the last pass
// leaves v[u R + q] = X[pos] with
//     pos = (b - j) R + j + q L,  b = t + T u,  j = b mod L,  L = N / R_last.
// Because L = N/R_last, pos = t + T (u + q E/R), so the forward output is already in the input
// order of an inverse transform after the register permutation u R + q -> u + q E/R.
#pragma once
#include "fft.cuh"

namespace tdgl {
namespace rf {

template <int N_, int E_, int R0_, int R1_ = 1, int R2_ = 1> struct Shape {
    static constexpr int N = N_, E = E_, T = N_ / E_, R0 = R0_, R1 = R1_, R2 = R2_;
    static constexpr int NP = R2_ > 1 ? 3 : (R1_ > 1 ? 2 : 1);
    static_assert(R0_ * R1_ * R2_ == N_, "the radices must multiply to N");
    static_assert(E_ % R0_ == 0 && E_ % R1_ == 0 && E_ % R2_ == 0, "every radix must divide E");
    static_assert(N_ % E_ == 0, "E must divide N");
};

// default shapes: 16 elements per thread for the power-of-two lengths, 12 for 3 * 2^k (radix 6 or
// 12 first: a prime-factor butterfly, so the first pass has no twiddle factors at all)
template <int N> struct Cfg;
template <> struct Cfg<16>  : Shape<16, 16, 16> {};
template <> struct Cfg<32>  : Shape<32, 16, 16, 2> {};
template <> struct Cfg<64>  : Shape<64, 16, 16, 4> {};
template <> struct Cfg<128> : Shape<128, 16, 16, 8> {};
template <> struct Cfg<256> : Shape<256, 16, 16, 16> {};
template <> struct Cfg<512> : Shape<512, 16, 16, 16, 2> {};
template <> struct Cfg<48>  : Shape<48, 12, 4, 4, 3> {};
template <> struct Cfg<96>  : Shape<96, 12, 6, 4, 4> {};
template <> struct Cfg<192> : Shape<192, 12, 12, 4, 4> {};

template <int N> __host__ __device__ constexpr int threads_per_line() { return Cfg<N>::T; }

template <class S> __host__ __device__ constexpr int radix(int p) {
    return p == 0 ? S::R0 : (p == 1 ? S::R1 : S::R2);
}
template <class S> __host__ __device__ constexpr int span_before(int p) {   // L of pass p
    return p == 0 ? 1 : (p == 1 ? S::R0 : S::R0 * S::R1);
}

// one pass on registers: v holds the inputs of this thread's butterflies in the order
// v[u + r E/R]; on return v[u R + q] holds output q of butterfly u
template <class S, int P, bool INV>
__device__ __forceinline__ void pass_regs(float2 (&v)[S::E], int t, const float2 *__restrict__ tw) {
    constexpr int E = S::E, T = S::T, N = S::N, R = radix<S>(P), L = span_before<S>(P), U = E / R;
    float2 o[E];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int b = t + T * u;
        const int j = b % L;
        float2 a[R];
#pragma unroll
        for (int r = 0; r < R; ++r) a[r] = v[u + r * U];
        if (L > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                float2 w = tw[r * j * (N / (L * R))];
                if (INV) w.y = -w.y;
                a[r] = cmul(a[r], w);
            }
        }
        dft<R, INV>(a);
#pragma unroll
        for (int q = 0; q < R; ++q) o[u * R + q] = a[q];
    }
#pragma unroll
    for (int i = 0; i < E; ++i) v[i] = o[i];
}

// position of output register i = u R + q after pass P
template <class S, int P>
__device__ __forceinline__ int out_pos(int t, int i) {
    constexpr int T = S::T, R = radix<S>(P), L = span_before<S>(P);
    const int u = i / R, q = i % R;
    const int b = t + T * u;
    const int j = b % L;
    return (b - j) * R + j + q * L;
}

// input position of register i = u + r E/R before pass P
template <class S, int P>
__device__ __forceinline__ int in_pos(int t, int i) {
    constexpr int T = S::T, R = radix<S>(P), U = S::E / R;
    const int u = i % U, r = i / U;
    return t + T * u + r * (S::N / R);
}

// exchange through shared memory: write outputs of pass P, read inputs of pass P+1
template <class S, int P, class Idx>
__device__ __forceinline__ void exchange(float2 (&v)[S::E], int t, float2 *X, Idx idx) {
#pragma unroll
    for (int i = 0; i < S::E; ++i) X[idx(out_pos<S, P>(t, i))] = v[i];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < S::E; ++i) v[i] = X[idx(in_pos<S, P + 1>(t, i))];
    __syncthreads();
}

// Full transform of shape S.  All threads of the block must call it (it synchronizes).  On
// return v[i] = X[final_pos<S>(t, i)].
template <class S, bool INV, class Idx>
__device__ __forceinline__ void fft(float2 (&v)[S::E], int t, float2 *X, Idx idx, const float2 *__restrict__ tw) {
    pass_regs<S, 0, INV>(v, t, tw);
    if constexpr (S::NP > 1) {
        exchange<S, 0>(v, t, X, idx);
        pass_regs<S, 1, INV>(v, t, tw);
    }
    if constexpr (S::NP > 2) {
        exchange<S, 1>(v, t, X, idx);
        pass_regs<S, 2, INV>(v, t, tw);
    }
}

template <class S>
__device__ __forceinline__ int final_pos(int t, int i) { return out_pos<S, S::NP - 1>(t, i); }

// Three transforms of shape S at once (three independent vectors held by the same threads, each
// with its own exchange buffer): the passes run back to back on the three vectors and every
// exchange serves all three, so a block waits at a third of the barriers and each thread has three
// independent butterflies in flight per pass.  Same results as three calls of fft.
template <class S, int P, class Idx>
__device__ __forceinline__ void exchange3(float2 (&a)[S::E], float2 (&b)[S::E], float2 (&c)[S::E], int t,
                                          float2 *Xa, float2 *Xb, float2 *Xc, Idx idx) {
#pragma unroll
    for (int i = 0; i < S::E; ++i) {
        const int q = idx(out_pos<S, P>(t, i));
        Xa[q] = a[i];
        Xb[q] = b[i];
        Xc[q] = c[i];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < S::E; ++i) {
        const int q = idx(in_pos<S, P + 1>(t, i));
        a[i] = Xa[q];
        b[i] = Xb[q];
        c[i] = Xc[q];
    }
    __syncthreads();
}

template <class S, bool INV, class Idx>
__device__ __forceinline__ void fft3(float2 (&a)[S::E], float2 (&b)[S::E], float2 (&c)[S::E], int t, float2 *Xa,
                                     float2 *Xb, float2 *Xc, Idx idx, const float2 *__restrict__ tw) {
    pass_regs<S, 0, INV>(a, t, tw);
    pass_regs<S, 0, INV>(b, t, tw);
    pass_regs<S, 0, INV>(c, t, tw);
    if constexpr (S::NP > 1) {
        exchange3<S, 0>(a, b, c, t, Xa, Xb, Xc, idx);
        pass_regs<S, 1, INV>(a, t, tw);
        pass_regs<S, 1, INV>(b, t, tw);
        pass_regs<S, 1, INV>(c, t, tw);
    }
    if constexpr (S::NP > 2) {
        exchange3<S, 1>(a, b, c, t, Xa, Xb, Xc, idx);
        pass_regs<S, 2, INV>(a, t, tw);
        pass_regs<S, 2, INV>(b, t, tw);
        pass_regs<S, 2, INV>(c, t, tw);
    }
}

// Zero padding to at least twice the data length (N >= 2n): the input registers m >= E/2 hold
// positions t + T m >= N/2 >= n, which are zero, and the output registers i whose last-pass index
// q = i mod R (R the last radix) is >= R/2 hold positions (b - j) R + j + q N/R >= N/2, which are
// not kept.  These compile-time forms of facts the run-time bounds already imply let the compiler
// drop the arithmetic on known zeros and on discarded outputs.
template <class S> __host__ __device__ constexpr bool padded_in(int m) {
    return S::N % 2 != 0 || S::E % 2 != 0 || m < S::E / 2;
}
template <class S> __host__ __device__ constexpr bool kept_out(int i) {
    return radix<S>(S::NP - 1) % 2 != 0 || (i % radix<S>(S::NP - 1)) < radix<S>(S::NP - 1) / 2;
}

// register index holding X[t + T m] after a forward transform (inverse of final_pos within a thread)
template <class S>
__host__ __device__ constexpr int final_reg(int m) {
    return (m % (S::E / radix<S>(S::NP - 1))) * radix<S>(S::NP - 1) + m / (S::E / radix<S>(S::NP - 1));
}

}  // namespace rf
}  // namespace tdgl
