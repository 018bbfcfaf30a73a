// Length-specialized y and z passes of the zero-padded convolution (Eqs. 5-6), built on the
// register FFT of fft_reg.cuh.  Thread (t, l) of a block owns position t of line l (column kx0 + l,
// or, in an "across" item, row r0 + l of one column):
// for every register the 16 (or 8) lanes of a half-warp touch consecutive kx of one row, so all
// global loads and stores are full 64/128-byte segments and every shared-memory exchange
// (layout [pos][l]) is conflict-free.
#pragma once
#include "fft_reg.cuh"
#include "kernels.cuh"
#include "tc.cuh"

namespace tdgl {

// work item .w: line count, | kAcross when the lanes run over rows of one column instead of
// over columns of one row (the Nyquist column x = Mx/2)
constexpr int kAcross = 1 << 16;

template <int N> __host__ __device__ constexpr int lines_per_block() {
    return (256 / rf::threads_per_line<N>()) < 16 ? (256 / rf::threads_per_line<N>()) : 16;
}

// Shapes of the z pass, V = radix-schedule variant (picked per length by the host's autotuner):
//   V = 0: the default shapes (16 elements per thread; radices 16 8 for 128, 16 16 for 256,
//          16 16 2 for 512), 128-thread blocks;
//   V = 1: for 128, 256 and 512 points 8 elements per thread (radices 8 8 2, 8 8 4, 8 8 8): half
//          the registers, 256-thread blocks with the same lines and shared memory, so an SM holds
//          twice the warps, at the price of one more exchange.
//   V = 2: for 128 and 256 points the shape of V = 1, plus the block's rows of the tensor table staged
//          in shared memory by one TMA copy per component pair at the start, so that their
//          latency overlaps the forward transforms instead of stalling the multiply (three
//          blocks per SM instead of four).
//   V = 3: V = 2 with the three components transformed together (k_zpass3): each pass runs on the
//          three components back to back and each exchange serves all three (a third of the
//          barriers, three independent butterflies per thread), and the 3x3 multiply works on
//          registers only.
// All variants give every length the same lines per block, hence the same work items.
template <int N, int V> struct ZCfg : rf::Cfg<N> {};
template <> struct ZCfg<128, 1> : rf::Shape<128, 8, 8, 8, 2> {};
template <> struct ZCfg<128, 2> : ZCfg<128, 1> {};
template <> struct ZCfg<256, 1> : rf::Shape<256, 8, 8, 8, 4> {};
template <> struct ZCfg<512, 1> : rf::Shape<512, 8, 8, 8, 8> {};
template <> struct ZCfg<256, 2> : ZCfg<256, 1> {};
template <> struct ZCfg<128, 3> : ZCfg<128, 1> {};
template <> struct ZCfg<256, 3> : ZCfg<256, 1> {};
// variant V stages the tensor rows in shared memory
template <int V> __host__ __device__ constexpr bool zstaged() { return V == 2 || V == 3; }
template <int N, int V> __host__ __device__ constexpr int zthreads() { return ZCfg<N, V>::E == 8 ? 256 : 128; }
template <int N, int V> __host__ __device__ constexpr int zlines_per_block() {
    return (zthreads<N, V>() / ZCfg<N, V>::T) < 16 ? (zthreads<N, V>() / ZCfg<N, V>::T) : 16;
}
static_assert(zlines_per_block<128, 0>() == zlines_per_block<128, 1>() &&
                  zlines_per_block<256, 0>() == zlines_per_block<256, 1>() &&
                  zlines_per_block<512, 0>() == zlines_per_block<512, 1>(),
              "z-pass variants must share the work items");

// y transform of the x-spectrum: forward (ny -> My, zero padded) or inverse (My -> first ny)
template <int N, bool INV>
__global__ void __launch_bounds__(256) k_ypass(const SimDev *__restrict__ sims, const int4 *__restrict__ items) {
    constexpr int E = rf::Cfg<N>::E, T = N / E, KX = lines_per_block<N>();
    __shared__ float2 S[N * KX];
    __shared__ float2 tw[N];
    const int4 it = items[blockIdx.x];
    const SimDev &D = sims[it.x];
    if (D.skip) return;   // a batch member that has left the relaxation
    const bool across = (it.w & kAcross) != 0;
    const int cnt = it.w & (kAcross - 1);
    const int l = threadIdx.x % KX, t = threadIdx.x / KX;
    const int cz = across ? it.y + l : it.y, kx = across ? it.z : it.z + l;   // this lane's line
    const bool ok = l < cnt;
    for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = D.tw[D.py.tw + i];
    const int ny = D.ny, kxp = D.kxp;
    float2 v[E];
    if (!INV) {
        const float2 *src = D.X + (long)cz * ny * kxp + kx;
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int y = t + T * m;
            v[m] = (rf::padded_in<rf::Cfg<N>>(m) && ok && y < ny) ? src[(long)y * kxp] : make_float2(0.f, 0.f);
        }
    } else {
        const float2 *src = D.Y + (long)cz * N * kxp + kx;
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = ok ? src[(long)(t + T * m) * kxp] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    rf::fft<rf::Cfg<N>, INV>(v, t, S, [&](int pos) { return pos * KX + l; }, tw);
    if (!ok) return;
    if (!INV) {
        float2 *dst = D.Y + (long)cz * N * kxp + kx;
#pragma unroll
        for (int i = 0; i < E; ++i) dst[(long)rf::final_pos<rf::Cfg<N>>(t, i) * kxp] = v[i];
    } else {
        float2 *dst = D.X + (long)cz * ny * kxp + kx;
#pragma unroll
        for (int i = 0; i < E; ++i) {
            const int y = rf::final_pos<rf::Cfg<N>>(t, i);
            if (rf::kept_out<rf::Cfg<N>>(i) && y < ny) dst[(long)y * kxp] = v[i];
        }
    }
}

// rows per component pair of the staged tensor tile (N/2 + 1 values of kz for each of the KX
// columns), rounded up so that every pair starts on a 128-byte boundary
template <int N, int KX> __host__ __device__ constexpr int ztile_rows() {
    return ((N / 2 + 1) * KX * (int)sizeof(float2) + 127) / 128 * 128 / (KX * (int)sizeof(float2));
}
// dynamic shared memory of k_zpass: three component spectra [3][N][KX], the twiddles and (staged
// variants) the tensor tile [3][rows][KX], plus slack to start the spectra on a 128-byte boundary
// (the alignment of a TMA destination)
template <int N, int V> __host__ __device__ constexpr size_t zpass_smem() {
    constexpr int KX = zlines_per_block<N, V>();
    return (3 * N * KX + N + (zstaged<V>() ? 3 * ztile_rows<N, KX>() * KX : 0)) * sizeof(float2) + 128;
}

// Row of position pos in a [N][KX] exchange buffer.  With KX < 16 lines a half-warp covers
// G = 16/KX positions; the first pass writes positions R0 apart, which would all start in the
// same bank.  Rows inside each aligned group of G are permuted by (pos / R0) mod G, which
// spreads those writes over G different bank groups and keeps consecutive positions (every
// other access) in distinct bank groups too.
template <int N, int V, int KX> __device__ __forceinline__ int zrow(int pos) {
    constexpr int G = KX >= 16 ? 1 : 16 / KX, R0 = ZCfg<N, V>::R0;
    static_assert(G == 1 || (R0 % G == 0 && (G & (G - 1)) == 0), "swizzle group must divide the first radix");
    if constexpr (G == 1) return pos;
    else return pos ^ ((pos / R0) & (G - 1));
}

// z transform, per-k 3x3 tensor multiply, inverse z transform (first nz outputs kept).
// The three components' inputs are copied asynchronously into shared memory, one commit group
// each, so the x transform starts while y and z are still in flight.  The forward spectra of x
// and y are parked in shared memory (each thread's own slots); z stays in registers through the
// multiply and its inverse runs first, straight from registers.
template <int N, int V>
__global__ void __launch_bounds__(zthreads<N, V>(), zstaged<V>() ? 3 : 4)
    k_zpass(const SimDev *__restrict__ sims, const int4 *__restrict__ items) {
    using S = ZCfg<N, V>;
    constexpr int E = S::E, T = S::T, KX = zlines_per_block<N, V>(), NR = ztile_rows<N, KX>();
    extern __shared__ float4 smem4[];
    float2 *A = reinterpret_cast<float2 *>((reinterpret_cast<uintptr_t>(smem4) + 127) & ~uintptr_t(127));   // [3][N][KX]
    float2 *tw = A + 3 * N * KX;                          // [N]
    float2 *Nt = tw + N;                                  // [3][NR][KX] staged tensor rows (V = 2)
    static_assert(!zstaged<V>() || ((3 * N * KX + N) * sizeof(float2)) % 128 == 0, "staged tile must start on 128 bytes");
    const int4 it = items[blockIdx.x];
    const SimDev &D = sims[it.x];
    if (D.skip) return;   // a batch member that has left the relaxation
    const bool across = (it.w & kAcross) != 0;
    const int cnt = it.w & (kAcross - 1);
    const int l = threadIdx.x % KX, t = threadIdx.x / KX;
    const int ky = across ? it.y + l : it.y, kx = across ? it.z : it.z + l;   // this lane's line
    const bool ok = l < cnt;
    const int nz = D.nz, My = D.My, kxp = D.kxp;
    const long zs = (long)My * kxp, cs = (long)nz * zs;
    const float2 *src = D.Y + (long)ky * kxp + kx;
    auto idx = [&](int pos) { return zrow<N, V, KX>(pos) * KX + l; };   // exchange layout
    // the reduced tensor rows this lane multiplies by (reflection signs for ky > My/2)
    const int kyr = (ky <= My / 2) ? ky : My - ky;
    const float sy = (ky <= My / 2) ? 1.f : -1.f;
    auto at = [&](int z) { return z * KX + l; };                          // input layout [z][line]
    // inputs of all three components in flight at once, component c on its own barrier / group:
    // regular items with one TMA copy per component (the z lines of KX columns), the Nyquist items
    // (lanes over ky) with 8-byte copies into each thread's own slots
    // (staged variant) the block's tensor rows follow on barrier 3: (kz = 0 .. N/2, kyr, its KX
    // columns) of each component pair
    __shared__ uint64_t zbar[4];
    // (the TMA destinations A + c N KX must be 128-byte aligned; checked, else the per-lane copies)
    const bool tma = D.has_ymap && !across && (tc::saddr(A) & 127u) == 0u;
    const bool staged = zstaged<V>() && tma && D.has_nmap;
    if (tma) {
        if (threadIdx.x == 0) {
            for (int c = 0; c < 4; ++c) tc::mbar_init(&zbar[c], 1);
            tc::mbar_fence_init();
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int c = 0; c < 3; ++c) {
                tc::mbar_expect_tx(&zbar[c], (uint32_t)(nz * KX * sizeof(float2)));
                tc::tma_load_4d(tc::saddr(A + c * N * KX), &D.ymap, &zbar[c], 2 * it.z, ky, 0, c);
            }
            if (staged) {
                tc::mbar_expect_tx(&zbar[3], (uint32_t)(3 * (N / 2 + 1) * KX * sizeof(float2)));
                for (int p = 0; p < 3; ++p) tc::tma_load_4d(tc::saddr(Nt + p * NR * KX), &D.nmap, &zbar[3], 2 * it.z, kyr, 0, p);
            }
        }
    } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            if (ok) {
#pragma unroll
                for (int m = 0; m < E; ++m) {
                    const int z = t + T * m;
                    if (z < nz) {
                        const unsigned dst = (unsigned)__cvta_generic_to_shared(A + c * N * KX + at(z));
                        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(src + c * cs + z * zs));
                    }
                }
            }
            asm volatile("cp.async.commit_group;\n" ::);
        }
    }
    // component c's inputs have landed (for this thread's slots, or for the whole TMA box)
    auto arrived = [&](int c) {
        if (tma) {
            if (!tc::mbar_wait(&zbar[c], 0u, 1L << 24) && threadIdx.x == 0) atomicOr(D.flag, 2);
        } else if (c == 0) {
            asm volatile("cp.async.wait_group 2;\n" ::);
        } else if (c == 1) {
            asm volatile("cp.async.wait_group 1;\n" ::);
        } else {
            asm volatile("cp.async.wait_group 0;\n" ::);
        }
    };
    const long ns = (long)D.kzh * D.kyh * kxp;
    const float2 *Nb = D.Nhat + (long)kyr * kxp + kx;
    const long rowN = (long)D.kyh * kxp;
    for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = D.tw[D.pz.tw + i];
    // forward transform of component c from this thread's own input slots; Ac is its exchange buffer
    auto forward = [&](int c, float2(&v)[E]) {
        float2 *Ac = A + c * N * KX;
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int z = t + T * m;
            v[m] = (rf::padded_in<S>(m) && ok && z < nz) ? Ac[at(z)] : make_float2(0.f, 0.f);
        }
        __syncthreads();   // inputs (and the twiddles) read before the exchanges overwrite them
        rf::fft<S, false>(v, t, Ac, idx, tw);
    };
    {
        arrived(0);
        float2 v[E];
        forward(0, v);
#pragma unroll
        for (int i = 0; i < E; ++i) A[idx(rf::final_pos<S>(t, i))] = v[i];
    }
    {
        arrived(1);
        float2 v[E];
        forward(1, v);
#pragma unroll
        for (int i = 0; i < E; ++i) A[N * KX + idx(rf::final_pos<S>(t, i))] = v[i];
    }
    arrived(2);
    float2 w[E];
    forward(2, w);
    if (staged && !tc::mbar_wait(&zbar[3], 0u, 1L << 24) && threadIdx.x == 0) atomicOr(D.flag, 2);
    // E-hat(k) = escale * N-hat(k) P-hat(k); N-hat from the reduced table with reflection signs.
    // x and y results go back to their owner's slots, z stays in w.
    const float es = D.escale;
#pragma unroll
    for (int i = 0; i < E; ++i) {
        const int kz = rf::final_pos<S>(t, i);
        const int kzr = (kz <= N / 2) ? kz : N - kz;
        const float sz = (kz <= N / 2) ? 1.f : -1.f;
        const float2 *Np = Nb + kzr * rowN;
        float nxx = 0.f, nyy = 0.f, nzz = 0.f, nxy = 0.f, nxz = 0.f, nyz = 0.f;
        if (staged) {
            const float2 *Nl = Nt + kzr * KX + l;
            const float2 n0 = Nl[0], n1 = Nl[NR * KX], n2 = Nl[2 * NR * KX];
            nxx = n0.x; nyy = n0.y; nzz = n1.x;
            nxy = sy * n1.y; nxz = sz * n2.x; nyz = sy * sz * n2.y;
        } else if (ok) {
            const float2 n0 = __ldg(Np), n1 = __ldg(Np + ns), n2 = __ldg(Np + 2 * ns);
            nxx = n0.x; nyy = n0.y; nzz = n1.x;
            nxy = sy * n1.y; nxz = sz * n2.x; nyz = sy * sz * n2.y;
        }
        const int p = idx(kz);
        const float2 px = A[p], py = A[N * KX + p], pz = w[i];
        A[p] = make_float2(es * (nxx * px.x + nxy * py.x + nxz * pz.x), es * (nxx * px.y + nxy * py.y + nxz * pz.y));
        A[N * KX + p] = make_float2(es * (nxy * px.x + nyy * py.x + nyz * pz.x), es * (nxy * px.y + nyy * py.y + nyz * pz.y));
        w[i] = make_float2(es * (nxz * px.x + nyz * py.x + nzz * pz.x), es * (nxz * px.y + nyz * py.y + nzz * pz.y));
    }
    float2 *dst = D.Y + (long)ky * kxp + kx;
    // component c's first nz outputs back into Y.  Regular items: into its exchange buffer (free
    // once its inverse has returned) in the layout of the input box, then one TMA store of the box
    // (in a partial item the columns past the count fall into Y's padding, which nothing reads);
    // Nyquist items: 8-byte stores from each lane.
    auto store = [&](int c, const float2(&v)[E]) {
        if (tma) {
            float2 *Ac = A + c * N * KX;
#pragma unroll
            for (int i = 0; i < E; ++i) {
                const int z = rf::final_pos<S>(t, i);
                if (rf::kept_out<S>(i) && z < nz) Ac[at(z)] = v[i];
            }
            tc::fence_proxy_async();   // the box's generic-proxy writes before the copy reads it
            __syncthreads();
            if (threadIdx.x == 0) {
                tc::tma_store_4d(&D.ymap, tc::saddr(Ac), 2 * it.z, ky, 0, c);
                tc::bulk_commit();
            }
        } else if (ok) {
#pragma unroll
            for (int i = 0; i < E; ++i) {
                const int z = rf::final_pos<S>(t, i);
                if (rf::kept_out<S>(i) && z < nz) dst[c * cs + z * zs] = v[i];
            }
        }
    };
    {
        // z first: inverse input order is the forward output order after the register permutation;
        // its exchange buffer is the z region, which nothing reads any more
        float2 v[E];
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = w[rf::final_reg<S>(m)];
        rf::fft<S, true>(v, t, A + 2 * N * KX, idx, tw);
        store(2, v);
    }
#pragma unroll 1
    for (int c = 0; c < 2; ++c) {
        float2 *Ac = A + c * N * KX;
        float2 v[E];
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = Ac[idx(t + T * m)];
        __syncthreads();   // every slot of Ac read by its owner before the exchanges overwrite it
        rf::fft<S, true>(v, t, Ac, idx, tw);
        store(c, v);
    }
    if (tma && threadIdx.x == 0) tc::bulk_wait_read_all();   // the boxes read before shared memory goes
}


// Variant 3 of the z pass: the three components' transforms run together (rf::fft3).  Work items,
// input and output layouts, the staged tensor rows and the Nyquist items are those of k_zpass<N, 2>.
template <int N>
__global__ void __launch_bounds__(zthreads<N, 3>(), 2)
    k_zpass3(const SimDev *__restrict__ sims, const int4 *__restrict__ items) {
    using S = ZCfg<N, 3>;
    constexpr int E = S::E, T = S::T, KX = zlines_per_block<N, 3>(), NR = ztile_rows<N, KX>();
    extern __shared__ float4 smem4[];
    float2 *A = reinterpret_cast<float2 *>((reinterpret_cast<uintptr_t>(smem4) + 127) & ~uintptr_t(127));   // [3][N][KX]
    float2 *tw = A + 3 * N * KX;                          // [N]
    float2 *Nt = tw + N;                                  // [3][NR][KX] staged tensor rows
    float2 *A0 = A, *A1 = A + N * KX, *A2 = A + 2 * N * KX;
    const int4 it = items[blockIdx.x];
    const SimDev &D = sims[it.x];
    if (D.skip) return;   // a batch member that has left the relaxation
    const bool across = (it.w & kAcross) != 0;
    const int cnt = it.w & (kAcross - 1);
    const int l = threadIdx.x % KX, t = threadIdx.x / KX;
    const int ky = across ? it.y + l : it.y, kx = across ? it.z : it.z + l;   // this lane's line
    const bool ok = l < cnt;
    const int nz = D.nz, My = D.My, kxp = D.kxp;
    const long zs = (long)My * kxp, cs = (long)nz * zs;
    const float2 *src = D.Y + (long)ky * kxp + kx;
    int *const flag = D.flag;
    auto idx = [&](int pos) { return zrow<N, 3, KX>(pos) * KX + l; };
    const int kyr = (ky <= My / 2) ? ky : My - ky;
    const float sy = (ky <= My / 2) ? 1.f : -1.f;
    auto at = [&](int z) { return z * KX + l; };
    __shared__ uint64_t zbar[4];
    const bool tma = D.has_ymap && !across && (tc::saddr(A) & 127u) == 0u;
    const bool staged = tma && D.has_nmap;
    if (tma) {
        if (threadIdx.x == 0) {
            for (int c = 0; c < 4; ++c) tc::mbar_init(&zbar[c], 1);
            tc::mbar_fence_init();
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int c = 0; c < 3; ++c) {
                tc::mbar_expect_tx(&zbar[c], (uint32_t)(nz * KX * sizeof(float2)));
                tc::tma_load_4d(tc::saddr(A + c * N * KX), &D.ymap, &zbar[c], 2 * it.z, ky, 0, c);
            }
            if (staged) {
                tc::mbar_expect_tx(&zbar[3], (uint32_t)(3 * (N / 2 + 1) * KX * sizeof(float2)));
                for (int p = 0; p < 3; ++p) tc::tma_load_4d(tc::saddr(Nt + p * NR * KX), &D.nmap, &zbar[3], 2 * it.z, kyr, 0, p);
            }
        }
    } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            if (ok) {
#pragma unroll
                for (int m = 0; m < E; ++m) {
                    const int z = t + T * m;
                    if (z < nz) {
                        const unsigned dst = (unsigned)__cvta_generic_to_shared(A + c * N * KX + at(z));
                        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(src + c * cs + z * zs));
                    }
                }
            }
        }
        asm volatile("cp.async.commit_group;\n" ::);
    }
    for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = D.tw[D.pz.tw + i];
    if (tma) {
        for (int c = 0; c < 3; ++c)
            if (!tc::mbar_wait(&zbar[c], 0u, 1L << 24) && threadIdx.x == 0) atomicOr(flag, 2);
    } else {
        asm volatile("cp.async.wait_group 0;\n" ::);
    }
    // forward transforms of the three components from this thread's own input slots
    float2 a[E], b[E], c[E];
#pragma unroll
    for (int m = 0; m < E; ++m) {
        const int z = t + T * m;
        const bool in = rf::padded_in<S>(m) && ok && z < nz;
        a[m] = in ? A0[at(z)] : make_float2(0.f, 0.f);
        b[m] = in ? A1[at(z)] : make_float2(0.f, 0.f);
        c[m] = in ? A2[at(z)] : make_float2(0.f, 0.f);
    }
    __syncthreads();   // inputs (and the twiddles) read before the exchanges overwrite them
    rf::fft3<S, false>(a, b, c, t, A0, A1, A2, idx, tw);
    if (staged && !tc::mbar_wait(&zbar[3], 0u, 1L << 24) && threadIdx.x == 0) atomicOr(flag, 2);
    // E-hat(k) = escale * N-hat(k) P-hat(k) in registers, then the inverse transforms' input order
    const float es = D.escale;
    const long ns = (long)D.kzh * D.kyh * kxp;
    const float2 *Nb = D.Nhat + (long)kyr * kxp + kx;
    const long rowN = (long)D.kyh * kxp;
#pragma unroll
    for (int i = 0; i < E; ++i) {
        const int kz = rf::final_pos<S>(t, i);
        const int kzr = (kz <= N / 2) ? kz : N - kz;
        const float sz = (kz <= N / 2) ? 1.f : -1.f;
        float nxx = 0.f, nyy = 0.f, nzz = 0.f, nxy = 0.f, nxz = 0.f, nyz = 0.f;
        if (staged) {
            const float2 *Nl = Nt + kzr * KX + l;
            const float2 n0 = Nl[0], n1 = Nl[NR * KX], n2 = Nl[2 * NR * KX];
            nxx = n0.x; nyy = n0.y; nzz = n1.x;
            nxy = sy * n1.y; nxz = sz * n2.x; nyz = sy * sz * n2.y;
        } else if (ok) {
            const float2 *Np = Nb + kzr * rowN;
            const float2 n0 = __ldg(Np), n1 = __ldg(Np + ns), n2 = __ldg(Np + 2 * ns);
            nxx = n0.x; nyy = n0.y; nzz = n1.x;
            nxy = sy * n1.y; nxz = sz * n2.x; nyz = sy * sz * n2.y;
        }
        const float2 px = a[i], py = b[i], pz = c[i];
        a[i] = make_float2(es * (nxx * px.x + nxy * py.x + nxz * pz.x), es * (nxx * px.y + nxy * py.y + nxz * pz.y));
        b[i] = make_float2(es * (nxy * px.x + nyy * py.x + nyz * pz.x), es * (nxy * px.y + nyy * py.y + nyz * pz.y));
        c[i] = make_float2(es * (nxz * px.x + nyz * py.x + nzz * pz.x), es * (nxz * px.y + nyz * py.y + nzz * pz.y));
    }
    float2 ia[E], ib[E], ic[E];
#pragma unroll
    for (int m = 0; m < E; ++m) {
        ia[m] = a[rf::final_reg<S>(m)];
        ib[m] = b[rf::final_reg<S>(m)];
        ic[m] = c[rf::final_reg<S>(m)];
    }
    // the exchange buffers are free: the last forward exchange's reads finished at its barrier
    rf::fft3<S, true>(ia, ib, ic, t, A0, A1, A2, idx, tw);
    // the first nz outputs back into Y: regular items through the input boxes and one TMA store per
    // component, Nyquist items with 8-byte stores from each lane
    if (tma) {
        // (every lane's reads of the last exchange finished at its closing barrier)
#pragma unroll
        for (int i = 0; i < E; ++i) {
            const int z = rf::final_pos<S>(t, i);
            if (rf::kept_out<S>(i) && z < nz) {
                A0[at(z)] = ia[i];
                A1[at(z)] = ib[i];
                A2[at(z)] = ic[i];
            }
        }
        tc::fence_proxy_async();
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int q = 0; q < 3; ++q) tc::tma_store_4d(&D.ymap, tc::saddr(A + q * N * KX), 2 * it.z, ky, 0, q);
            tc::bulk_commit();
            tc::bulk_wait_read_all();   // the boxes read before shared memory goes
        }
    } else if (ok) {
        float2 *dst = D.Y + (long)ky * kxp + kx;
#pragma unroll
        for (int i = 0; i < E; ++i) {
            const int z = rf::final_pos<S>(t, i);
            if (rf::kept_out<S>(i) && z < nz) {
                dst[z * zs] = ia[i];
                dst[cs + z * zs] = ib[i];
                dst[2 * cs + z * zs] = ic[i];
            }
        }
    }
}

}  // namespace tdgl
