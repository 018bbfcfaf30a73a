// Register-resident FFT of compile-time length N for groups of T = N/E threads per line.
//
// Each thread of a line holds E elements.  On entry thread t holds v[m] = x[t + T m]
// (m < E), which is exactly the input of the first Stockham pass (see fft.cuh for the pass
// definition): butterfly u of thread t is b = t + T u and reads elements b + r N/R_1, i.e.
// registers m = u + r E/R_1.  Between passes the outputs go through a shared-memory exchange
// buffer addressed by a caller functor idx(pos) (layout chosen by the caller for conflict-free,
// coalesced access); the last pass leaves v[u R + q] = X[pos] with
//     pos = (b - j) R + j + q L,  b = t + T u,  j = b mod L,  L = N / R_last.
// Because L = N/R_last, pos = t + T (u + q E/R), so the forward output is already in the input
// order of an inverse transform after the register permutation u R + q -> u + q E/R.
#pragma once
#include "fft.cuh"

namespace tdgl {
namespace rf {

template <int N> struct Cfg;
template <> struct Cfg<16>  { static constexpr int E = 16, NP = 1, R0 = 16, R1 = 1,  R2 = 1; };
template <> struct Cfg<32>  { static constexpr int E = 16, NP = 2, R0 = 16, R1 = 2,  R2 = 1; };
template <> struct Cfg<64>  { static constexpr int E = 16, NP = 2, R0 = 16, R1 = 4,  R2 = 1; };
template <> struct Cfg<128> { static constexpr int E = 16, NP = 2, R0 = 16, R1 = 8,  R2 = 1; };
template <> struct Cfg<256> { static constexpr int E = 16, NP = 2, R0 = 16, R1 = 16, R2 = 1; };
template <> struct Cfg<512> { static constexpr int E = 16, NP = 3, R0 = 16, R1 = 16, R2 = 2; };
template <> struct Cfg<48>  { static constexpr int E = 12, NP = 3, R0 = 4,  R1 = 4,  R2 = 3; };
template <> struct Cfg<96>  { static constexpr int E = 24, NP = 3, R0 = 8,  R1 = 4,  R2 = 3; };
template <> struct Cfg<192> { static constexpr int E = 24, NP = 3, R0 = 8,  R1 = 8,  R2 = 3; };

template <int N> __host__ __device__ constexpr int threads_per_line() { return N / Cfg<N>::E; }
template <int N> __host__ __device__ constexpr int radix(int p) {
    return p == 0 ? Cfg<N>::R0 : (p == 1 ? Cfg<N>::R1 : Cfg<N>::R2);
}
template <int N> __host__ __device__ constexpr int span_before(int p) {   // L of pass p
    return p == 0 ? 1 : (p == 1 ? Cfg<N>::R0 : Cfg<N>::R0 * Cfg<N>::R1);
}

// one pass on registers: v holds the inputs of this thread's butterflies in the order
// v[u + r E/R]; on return v[u R + q] holds output q of butterfly u
template <int N, int P, bool INV>
__device__ __forceinline__ void pass_regs(float2 (&v)[Cfg<N>::E], int t, const float2 *__restrict__ tw) {
    constexpr int E = Cfg<N>::E, T = N / E, R = radix<N>(P), L = span_before<N>(P), U = E / R;
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
template <int N, int P>
__device__ __forceinline__ int out_pos(int t, int i) {
    constexpr int E = Cfg<N>::E, T = N / E, R = radix<N>(P), L = span_before<N>(P);
    const int u = i / R, q = i % R;
    const int b = t + T * u;
    const int j = b % L;
    return (b - j) * R + j + q * L;
}

// input position of register i = u + r E/R before pass P
template <int N, int P>
__device__ __forceinline__ int in_pos(int t, int i) {
    constexpr int E = Cfg<N>::E, T = N / E, R = radix<N>(P), U = E / R;
    const int u = i % U, r = i / U;
    return t + T * u + r * (N / R);
}

// exchange through shared memory: write outputs of pass P, read inputs of pass P+1
template <int N, int P, class Idx>
__device__ __forceinline__ void exchange(float2 (&v)[Cfg<N>::E], int t, float2 *S, Idx idx) {
    constexpr int E = Cfg<N>::E;
#pragma unroll
    for (int i = 0; i < E; ++i) S[idx(out_pos<N, P>(t, i))] = v[i];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < E; ++i) v[i] = S[idx(in_pos<N, P + 1>(t, i))];
    __syncthreads();
}

// Full transform.  All threads of the block must call it (it synchronizes).  On return
// v[i] = X[final_pos<N>(t, i)].
template <int N, bool INV, class Idx>
__device__ __forceinline__ void fft(float2 (&v)[Cfg<N>::E], int t, float2 *S, Idx idx, const float2 *__restrict__ tw) {
    constexpr int NP = Cfg<N>::NP;
    pass_regs<N, 0, INV>(v, t, tw);
    if constexpr (NP > 1) {
        exchange<N, 0>(v, t, S, idx);
        pass_regs<N, 1, INV>(v, t, tw);
    }
    if constexpr (NP > 2) {
        exchange<N, 1>(v, t, S, idx);
        pass_regs<N, 2, INV>(v, t, tw);
    }
}

template <int N>
__device__ __forceinline__ int final_pos(int t, int i) { return out_pos<N, Cfg<N>::NP - 1>(t, i); }

// register index holding X[t + T m] after a forward transform (inverse of final_pos within a thread)
template <int N>
__host__ __device__ constexpr int final_reg(int m) {
    return (m % (Cfg<N>::E / radix<N>(Cfg<N>::NP - 1))) * radix<N>(Cfg<N>::NP - 1) +
           m / (Cfg<N>::E / radix<N>(Cfg<N>::NP - 1));
}

}  // namespace rf
}  // namespace tdgl
