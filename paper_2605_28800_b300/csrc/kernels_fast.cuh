// Length-specialized y and z passes of the zero-padded convolution (Eqs. 5-6), built on the
// register FFT of fft_reg.cuh.  Thread (t, l) of a block owns position t of line l (kx0 + l):
// for every register the 16 (or 8) lanes of a half-warp touch consecutive kx of one row, so all
// global loads and stores are full 64/128-byte segments and every shared-memory exchange
// (layout [pos][l]) is conflict-free.
#pragma once
#include "fft_reg.cuh"
#include "kernels.cuh"

namespace tdgl {

template <int N> __host__ __device__ constexpr int lines_per_block() {
    return (256 / rf::threads_per_line<N>()) < 16 ? (256 / rf::threads_per_line<N>()) : 16;
}
template <int N> __host__ __device__ constexpr int zlines_per_block() {
    return (128 / rf::threads_per_line<N>()) < 16 ? (128 / rf::threads_per_line<N>()) : 16;
}

// y transform of the x-spectrum: forward (ny -> My, zero padded) or inverse (My -> first ny)
template <int N, bool INV>
__global__ void __launch_bounds__(256) k_ypass(const SimDev *__restrict__ sims, const int4 *__restrict__ items) {
    constexpr int E = rf::Cfg<N>::E, T = N / E, KX = lines_per_block<N>();
    __shared__ float2 S[N * KX];
    __shared__ float2 tw[N];
    const int4 it = items[blockIdx.x];
    const SimDev &D = sims[it.x];
    const int cz = it.y, kx0 = it.z, cnt = it.w;
    const int l = threadIdx.x % KX, t = threadIdx.x / KX;
    const bool ok = l < cnt;
    for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = D.tw[D.py.tw + i];
    const int ny = D.ny, kxp = D.kxp;
    float2 v[E];
    if (!INV) {
        const float2 *src = D.X + (long)cz * ny * kxp + kx0 + l;
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int y = t + T * m;
            v[m] = (ok && y < ny) ? src[(long)y * kxp] : make_float2(0.f, 0.f);
        }
    } else {
        const float2 *src = D.Y + (long)cz * N * kxp + kx0 + l;
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = ok ? src[(long)(t + T * m) * kxp] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    rf::fft<N, INV>(v, t, S, [&](int pos) { return pos * KX + l; }, tw);
    if (!ok) return;
    if (!INV) {
        float2 *dst = D.Y + (long)cz * N * kxp + kx0 + l;
#pragma unroll
        for (int i = 0; i < E; ++i) dst[(long)rf::final_pos<N>(t, i) * kxp] = v[i];
    } else {
        float2 *dst = D.X + (long)cz * ny * kxp + kx0 + l;
#pragma unroll
        for (int i = 0; i < E; ++i) {
            const int y = rf::final_pos<N>(t, i);
            if (y < ny) dst[(long)y * kxp] = v[i];
        }
    }
}

// dynamic shared memory of k_zpass: three component spectra [3][N][KX] and the twiddles
template <int N> __host__ __device__ constexpr size_t zpass_smem() {
    return (3 * N * zlines_per_block<N>() + N) * sizeof(float2);
}

// z transform, per-k 3x3 tensor multiply, inverse z transform (first nz outputs kept).
// The three forward spectra are parked in shared memory (each thread's own slots) so that the
// block needs few registers and several blocks share an SM.
template <int N>
__global__ void __launch_bounds__(128, 4) k_zpass(const SimDev *__restrict__ sims, const int4 *__restrict__ items) {
    constexpr int E = rf::Cfg<N>::E, T = N / E, KX = zlines_per_block<N>();
    extern __shared__ float4 smem4[];
    float2 *A = reinterpret_cast<float2 *>(smem4);      // [3][N][KX]
    float2 *tw = A + 3 * N * KX;                          // [N]
    const int4 it = items[blockIdx.x];
    const SimDev &D = sims[it.x];
    const int ky = it.y, kx0 = it.z, cnt = it.w;
    const int l = threadIdx.x % KX, t = threadIdx.x / KX;
    const bool ok = l < cnt;
    for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = D.tw[D.pz.tw + i];
    const int nz = D.nz, My = D.My, kxp = D.kxp;
    const long zs = (long)My * kxp, cs = (long)nz * zs;
    const float2 *src = D.Y + (long)ky * kxp + kx0 + l;
    auto idx = [&](int pos) { return pos * KX + l; };
    // all three components' inputs in flight at once: asynchronous 8-byte copies into this
    // thread's own slots of the spectra buffers
    if (ok) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const int z = t + T * m;
                if (z < nz) {
                    const unsigned dst = (unsigned)__cvta_generic_to_shared(A + c * N * KX + idx(z));
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(src + c * cs + z * zs));
                }
            }
    }
    asm volatile("cp.async.commit_group;\n" ::);
    asm volatile("cp.async.wait_group 0;\n" ::);
    __syncthreads();
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
        float2 *Ac = A + c * N * KX;
        float2 v[E];
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int z = t + T * m;
            v[m] = (ok && z < nz) ? Ac[idx(z)] : make_float2(0.f, 0.f);
        }
        __syncthreads();   // own slots read before the exchanges overwrite them
        rf::fft<N, false>(v, t, Ac, idx, tw);
#pragma unroll
        for (int i = 0; i < E; ++i) Ac[idx(rf::final_pos<N>(t, i))] = v[i];
    }
    // E-hat(k) = escale * N-hat(k) P-hat(k) on this thread's own slots; N-hat from the reduced
    // table with reflection signs
    const int kyr = (ky <= My / 2) ? ky : My - ky;
    const float sy = (ky <= My / 2) ? 1.f : -1.f;
    const long ns = (long)D.kzh * D.kyh * D.Kx;
    const float es = D.escale;
    const float *Nb = D.Nhat + (long)kyr * D.Kx + kx0 + l;
    const long rowN = (long)D.kyh * D.Kx;
#pragma unroll 8
    for (int i = 0; i < E; ++i) {
        const int kz = rf::final_pos<N>(t, i);
        const int kzr = (kz <= N / 2) ? kz : N - kz;
        const float sz = (kz <= N / 2) ? 1.f : -1.f;
        const float *Np = Nb + kzr * rowN;
        float nxx = 0.f, nyy = 0.f, nzz = 0.f, nxy = 0.f, nxz = 0.f, nyz = 0.f;
        if (ok) {
            nxx = __ldg(Np); nyy = __ldg(Np + ns); nzz = __ldg(Np + 2 * ns);
            nxy = sy * __ldg(Np + 3 * ns); nxz = sz * __ldg(Np + 4 * ns); nyz = sy * sz * __ldg(Np + 5 * ns);
        }
        const int p = idx(kz);
        const float2 px = A[p], py = A[N * KX + p], pz = A[2 * N * KX + p];
        A[p] = make_float2(es * (nxx * px.x + nxy * py.x + nxz * pz.x), es * (nxx * px.y + nxy * py.y + nxz * pz.y));
        A[N * KX + p] = make_float2(es * (nxy * px.x + nyy * py.x + nyz * pz.x), es * (nxy * px.y + nyy * py.y + nyz * pz.y));
        A[2 * N * KX + p] = make_float2(es * (nxz * px.x + nyz * py.x + nzz * pz.x), es * (nxz * px.y + nyz * py.y + nzz * pz.y));
    }
    float2 *dst = D.Y + (long)ky * kxp + kx0 + l;
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
        float2 *Ac = A + c * N * KX;
        float2 v[E];
        __syncthreads();   // every slot of Ac read by its owner before the exchanges overwrite it
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = Ac[idx(t + T * m)];
        __syncthreads();
        rf::fft<N, true>(v, t, Ac, idx, tw);
        if (ok) {
#pragma unroll
            for (int i = 0; i < E; ++i) {
                const int z = rf::final_pos<N>(t, i);
                if (z < nz) dst[c * cs + z * zs] = v[i];
            }
        }
    }
}

}  // namespace tdgl
