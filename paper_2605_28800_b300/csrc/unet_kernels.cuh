// Kernels of the learned warm start (a 3D U-Net): BF16 tensor-core convolutions with FP32
// accumulation in tensor memory, and the memory-bound pieces around them.
//
// Activations are channels-last ("NDHWC": [voxel][channel], voxel = ((b Z + z) Y + y) X + x) in
// BF16, gradients flowing back are FP32.  A convolution is an implicit GEMM
//     Y[v][o] = sum_k A[v][k] W[o][k],   k = (tap, i) -> 8-channel groups g = tap * (Ci/8) + i/8,
// M = 128 voxels per CTA, N = a tile of output channels, K consumed 16 at a time (two groups).
// The weight-gradient GEMM swaps the roles: M = output channels, N = (tap, input channel),
// K = voxels, with both operands transposed to [channel][voxel] first.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

#include <cuda.h>

#include "philox.cuh"
#include "tc.cuh"

namespace tdgl {
namespace unet {

constexpr int kStages = 3;          // cp.async -> MMA pipeline depth
constexpr int kSub = 4;             // 16-wide K sub-chunks (one MMA each) per pipeline stage
constexpr long kSpin = 1L << 24;    // mbarrier polls before a wait is declared failed

// a stage: kSub A sub-tiles (128 rows x 32 bytes each), then kSub B sub-tiles (BN rows x 32 bytes)
template <int BN> __host__ __device__ constexpr uint32_t stage_bytes() { return kSub * (128u * 32u + (uint32_t)BN * 32u); }
template <int BN> __host__ __device__ constexpr uint32_t tmem_cols() { return BN < 32 ? 32u : (uint32_t)BN; }
// dynamic shared memory: the stage ring, barriers and the TMEM slot, padded so that at most
// 512 / tmem_cols CTAs fit on an SM (their TMEM allocations then always fit together)
template <int BN> __host__ __device__ constexpr uint32_t gemm_smem() {
    constexpr uint32_t need = kStages * stage_bytes<BN>() + 128u;
    constexpr uint32_t per_sm = 232448u;                       // 227 KB + the 1 KB reserve
    constexpr uint32_t fit = per_sm / (512u / tmem_cols<BN>() + 1u) + 1024u;
    return (need > fit ? need : fit) + 1024u;                  // + alignment slack
}

// Pipelined main loop shared by both GEMMs over nsub 16-wide K sub-chunks: load(j, a_smem, b_smem)
// fills the tiles of sub-chunk j with cp.async; a stage holds kSub sub-chunks; one thread issues
// their MMAs once every thread's copies landed; a stage is refilled after the MMAs that read it
// have committed.  Returns false (in every thread) if a barrier wait ran out; the caller then
// still drains and frees.
template <int BN, class Load>
__device__ __forceinline__ bool mainloop(Load load, int nsub, uint8_t *tiles, uint64_t *bar, uint32_t tmem, int *issued) {
    constexpr uint32_t ST = stage_bytes<BN>(), AB = kSub * 128u * 32u, BB = (uint32_t)BN * 32u;
    constexpr uint32_t idesc = tc::idesc_bf16(128, BN);
    const uint32_t base = tc::saddr(tiles);
    const int tid = threadIdx.x;
    const int nch = (nsub + kSub - 1) / kSub;
    auto load_stage = [&](int c) {
        const uint32_t st = base + (uint32_t)(c % kStages) * ST;
#pragma unroll
        for (int u = 0; u < kSub; ++u) {
            const int j = c * kSub + u;
            if (j < nsub) load(j, st + (uint32_t)u * 4096u, st + AB + (uint32_t)u * BB);
        }
    };
    bool ok = true;
    *issued = 0;
#pragma unroll
    for (int c = 0; c < kStages - 1; ++c) {
        if (c < nch) load_stage(c);
        tc::cp_commit();
    }
    for (int c = 0; c < nch; ++c) {
        const int cn = c + kStages - 1;
        if (cn < nch && ok) {
            if (cn >= kStages) ok = tc::mbar_wait(&bar[cn % kStages], (unsigned)((cn - kStages) / kStages) & 1u, kSpin);
            if (ok) load_stage(cn);
        }
        tc::cp_commit();
        tc::cp_wait<kStages - 1>();
        tc::fence_proxy_async();
        ok = !__syncthreads_or(!ok);
        if (!ok) break;
        if (tid == 0) {
            tc::fence_after();
            const uint32_t st = base + (uint32_t)(c % kStages) * ST;
#pragma unroll
            for (int u = 0; u < kSub; ++u) {
                const int j = c * kSub + u;
                if (j < nsub)
                    tc::mma_bf16(tmem, tc::sdesc(st + (uint32_t)u * 4096u), tc::sdesc(st + AB + (uint32_t)u * BB), idesc,
                                 j > 0 ? 1u : 0u);
            }
            tc::mma_commit(&bar[c % kStages]);
        }
        *issued = c + 1;
    }
    tc::cp_wait<0>();
    // the last stage issued: its barrier phase completes when its MMAs (and all before) finished
    if (*issued > 0) {
        const int c = *issued - 1;
        const bool done = tc::mbar_wait(&bar[c % kStages], (unsigned)(c / kStages) & 1u, kSpin);
        ok = ok && done;
    }
    tc::fence_after();
    return !__syncthreads_or(!ok);
}

// CTA prologue: barriers, TMEM allocation by warp 0; returns the TMEM base address
template <int BN>
__device__ __forceinline__ uint32_t prologue(uint64_t *bar, uint32_t *tslot) {
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) tc::mbar_init(&bar[s], 1);
        tc::mbar_fence_init();
    }
    if (threadIdx.x < 32) tc::tmem_alloc(tslot, tmem_cols<BN>());
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    return *tslot;
}

template <int BN>
__device__ __forceinline__ void epilogue_free(uint32_t tmem) {
    tc::fence_before();
    __syncthreads();
    if (threadIdx.x < 32) {
        tc::fence_after();
        tc::tmem_free(tmem, tmem_cols<BN>());
    }
}

struct ConvP {
    const __nv_bfloat16 *x;   // [nvox][Ci]
    const __nv_bfloat16 *w;   // [Co][G * 8]  (k-group g = tap * Ci/8 + i/8; G even, tail zero)
    const float *bias;        // [Co] or null
    void *y;                  // [nvox][Co], BF16 or FP32
    long nvox;
    int Z, Y, X, Ci, Co, ntap, G, relu, f32out;
    int *err;
    int ksplit;               // > 1: the K range is split over gridDim.z CTAs, each writing its partial
    float *part;              // [ksplit][nvox][Co] FP32 partial sums (ksplit > 1), added by k_splitk_sum
};

// Epilogue of one output voxel v and 16 channels co0 .. co0 + 15 (the accumulator row r): bias,
// activation, store.  With whole 8-channel groups (Co a multiple of 8, co0 + 16 <= Co, y on 16 bytes)
// the row goes out as 16-byte vector stores (two for BF16, four for FP32), else channel by channel.
__device__ __forceinline__ void store_row16(const ConvP &p, long v, int co0, const float (&r)[16]) {
    float a[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const int co = co0 + j < p.Co ? co0 + j : p.Co - 1;
        a[j] = r[j] + (p.bias ? p.bias[co] : 0.f);
        if (p.relu) a[j] = fmaxf(a[j], 0.f);
    }
    if (p.Co % 8 == 0 && co0 + 16 <= p.Co && (reinterpret_cast<uintptr_t>(p.y) & 15u) == 0) {
        if (p.f32out) {
            float4 *dst = reinterpret_cast<float4 *>(reinterpret_cast<float *>(p.y) + v * p.Co + co0);
#pragma unroll
            for (int q = 0; q < 4; ++q) dst[q] = make_float4(a[4 * q], a[4 * q + 1], a[4 * q + 2], a[4 * q + 3]);
        } else {
            alignas(16) __nv_bfloat16 b[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) b[j] = __float2bfloat16_rn(a[j]);
            uint4 *dst = reinterpret_cast<uint4 *>(reinterpret_cast<__nv_bfloat16 *>(p.y) + v * p.Co + co0);
            dst[0] = reinterpret_cast<const uint4 *>(b)[0];
            dst[1] = reinterpret_cast<const uint4 *>(b)[1];
        }
        return;
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const int co = co0 + j;
        if (co >= p.Co) break;
        if (p.f32out) reinterpret_cast<float *>(p.y)[v * p.Co + co] = a[j];
        else reinterpret_cast<__nv_bfloat16 *>(p.y)[v * p.Co + co] = __float2bfloat16_rn(a[j]);
    }
}

// Y = act(bias + conv(X, W)) for a 3x3x3 (ntap 27) or 1x1x1 (ntap 1) kernel, zero padding.  With
// p.ksplit > 1 CTA (x, y, z) sums only the z-th of ksplit equal ranges of K sub-chunks and stores
// that partial sum; k_splitk_sum adds the partials in split order and applies bias and activation
// (for layers with too few voxel tiles to fill the GPU)
template <int BN>
__global__ void __launch_bounds__(128) k_conv(ConvP p) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *tiles = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *bar = reinterpret_cast<uint64_t *>(tiles + kStages * stage_bytes<BN>());
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + kStages);
    const int tid = threadIdx.x, warp = tid >> 5;
    const long v = (long)blockIdx.x * 128 + tid;      // this thread's row: output voxel
    const int n0 = blockIdx.y * BN;
    const bool vok = v < p.nvox;
    int vx = 0, vy = 0, vz = 0;
    long vb = 0;
    if (vok) {
        long q = v;
        vx = (int)(q % p.X); q /= p.X;
        vy = (int)(q % p.Y); q /= p.Y;
        vz = (int)(q % p.Z); vb = q / p.Z;
    }
    const int cg = p.Ci >> 3;
    const int nsub_all = p.G / 2, per = (nsub_all + p.ksplit - 1) / p.ksplit, j0 = (int)blockIdx.z * per;
    const int nsub = nsub_all - j0 < per ? nsub_all - j0 : per;   // >= 1: the host leaves no split empty
    const uint32_t tmem = prologue<BN>(bar, tslot);
    auto load = [&](int cl, uint32_t a_s, uint32_t b_s) {
        const int c = cl + j0;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int g = 2 * c + h;
            const int tap = g / cg, c8 = g - tap * cg;
            int dz = 0, dy = 0, dx = 0;
            if (p.ntap == 27) { dz = tap / 9 - 1; dy = (tap / 3) % 3 - 1; dx = tap % 3 - 1; }
            const int sz = vz + dz, sy = vy + dy, sx = vx + dx;
            const bool ok = vok && tap < p.ntap && (unsigned)sz < (unsigned)p.Z && (unsigned)sy < (unsigned)p.Y &&
                            (unsigned)sx < (unsigned)p.X;
            const __nv_bfloat16 *src = ok ? p.x + ((((vb * p.Z + sz) * p.Y + sy) * p.X + sx) * p.Ci + c8 * 8) : p.x;
            tc::cp16(a_s + tc::tile_off(tid, h), src, ok);
        }
        for (int i = tid; i < 2 * BN; i += 128) {
            const int n = i >> 1, h = i & 1, co = n0 + n;
            const bool ok = co < p.Co;
            const __nv_bfloat16 *src = ok ? p.w + ((long)co * p.G + 2 * c + h) * 8 : p.w;
            tc::cp16(b_s + tc::tile_off(n, h), src, ok);
        }
    };
    int issued;
    const bool ok = mainloop<BN>(load, nsub, tiles, bar, tmem, &issued);   // sub-chunk j: groups 2j, 2j+1
    if (!ok) {
        if (tid == 0) atomicOr(p.err, 1);
    } else {
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 16) {
            float r[16];
            tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
            if (!vok) continue;
            if (p.ksplit > 1) {
                float *dst = p.part + ((long)blockIdx.z * p.nvox + v) * p.Co;
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    if (n0 + c0 + j < p.Co) dst[n0 + c0 + j] = r[j];
                continue;
            }
            store_row16(p, v, n0 + c0, r);
        }
    }
    epilogue_free<BN>(tmem);
}

// y[v][o] = act(bias[o] + sum over splits s = 0, 1, ... of part[s][v][o]), in that order
__global__ void k_splitk_sum(const float *__restrict__ part, int nsplit, long nvox, int Co, const float *__restrict__ bias,
                             int relu, int f32out, void *__restrict__ y) {
    const long n = nvox * Co;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        float a = 0.f;
        for (int s = 0; s < nsplit; ++s) a += part[(long)s * n + i];
        a += bias ? bias[i % Co] : 0.f;
        if (relu) a = fmaxf(a, 0.f);
        if (f32out) reinterpret_cast<float *>(y)[i] = a;
        else reinterpret_cast<__nv_bfloat16 *>(y)[i] = __float2bfloat16_rn(a);
    }
}

// ---- brick convolution: the input brick staged once, the 27 taps as descriptor offsets -----------
//
// A CTA owns 128 ZT output voxels: x0..x0+7 (core-matrix rows) by y0..y0+15 (row groups) in the ZT
// planes z0 .. z0 + ZT - 1 (ZT = 1 or 2; planes past the grid dropped).  Per 16-channel chunk of the
// input, two TMA loads bring the brick with its one-voxel halo, 10 x 18 x (ZT + 2) voxels, as two planes
// (channels 0-7 and 8-15 of the chunk) of 16-byte voxel records, x fastest (out-of-grid voxels read
// as zero), and two more bring the chunk's weights for all 27 taps as [half][tap][output channel]
// records.  For a tap (dz, dy, dx) and output plane zz the A operand is the brick read from a
// shifted start: row group g at ((1 + zz + dz) * 18 + g + 1 + dy) * 10 + 1 + dx records, rows 16
// bytes apart, so its descriptor keeps the stride-dimension offset 160 bytes (one brick row) and the
// leading-dimension offset one plane; the B operand of the tap is its slice of the weights, shared
// by the planes, whose accumulators sit side by side in tensor memory.  Two planes per CTA share
// one brick (4 instead of 2 x 3 halo planes) and one weight load, and each copy round trip feeds 54
// MMAs; one plane per CTA keeps twice the CTAs for grids too small to fill the GPU otherwise.  One elected thread drives the pipeline: TMA into a stage, wait for its bytes, the MMAs,
// commit to the stage's "empty" barrier, refill the stage once those MMAs are done.
constexpr int kBX = 10, kBY = 18;
// ZT output planes per CTA: the brick is ZT + 2 planes deep; voxel records per 8-channel plane
// of the brick, and its bytes padded to 128
template <int ZT> __host__ __device__ constexpr int brick_records() { return kBX * kBY * (ZT + 2); }
template <int ZT> __host__ __device__ constexpr uint32_t brick_plane() { return (brick_records<ZT>() * 16u + 127u) / 128u * 128u; }
// the ZT planes' accumulators sit side by side in tensor memory
template <int BN, int ZT> __host__ __device__ constexpr uint32_t brick_tmem_cols() { return ZT * BN < 32 ? 32u : (uint32_t)(ZT * BN); }
template <int BN> __host__ __device__ constexpr uint32_t brick_wplane() { return 27u * BN * 16u; }
template <int BN, int ZT> __host__ __device__ constexpr uint32_t brick_stage_bytes() {
    return 2u * brick_plane<ZT>() + 2u * brick_wplane<BN>();
}
// S pipeline stages: 1 when the input has a single 16-channel chunk, 2 otherwise
template <int BN, int S, int ZT> __host__ __device__ constexpr uint32_t brick_smem() {
    return S * brick_stage_bytes<BN, ZT>() + 256u + 1024u;
}

// shared-memory descriptor with explicit leading / stride byte offsets
__device__ __forceinline__ uint64_t sdesc_lbo_sbo(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

struct BrickP {
    ConvP c;
    CUtensorMap tx;   // activations [B][Z][Y][X][Ci] BF16 as (Ci, X, Y, Z, B), box (8, 10, 18, ZT + 2, 1)
    CUtensorMap tw;   // weights [27][Co][Ci] BF16 as (Ci, Co, 27), box (8, BN, 27)
};

template <int BN, int S, int ZT>
__global__ void __launch_bounds__(128) k_conv_brick(const __grid_constant__ BrickP bp) {
    const ConvP &p = bp.c;
    constexpr uint32_t kPlane = brick_plane<ZT>();
    constexpr uint32_t ST = brick_stage_bytes<BN, ZT>(), AB = 2u * kPlane, WP = brick_wplane<BN>();
    constexpr uint32_t idesc = tc::idesc_bf16(128, BN);
    constexpr uint32_t kBytes = 2u * (uint32_t)brick_records<ZT>() * 16u + 2u * 27u * BN * 16u;   // per stage
    extern __shared__ uint8_t smem_raw[];
    uint8_t *tiles = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *full = reinterpret_cast<uint64_t *>(tiles + S * ST);
    uint64_t *empty = full + S;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(empty + S);
    int *s_state = reinterpret_cast<int *>(tslot + 2);     // [0] MMA stages issued, [1] ok
    const int tid = threadIdx.x, warp = tid >> 5;
    const int nbx = p.X / 8, nby = p.Y / 16, nzp = (p.Z + ZT - 1) / ZT;
    long q = blockIdx.x;
    const int bx = (int)(q % nbx); q /= nbx;
    const int by = (int)(q % nby); q /= nby;
    const int z0 = ZT * (int)(q % nzp);           // planes z0 .. z0 + ZT - 1 (the last ones may lie past Z)
    const int b = (int)(q / nzp);
    const int x0 = bx * 8, y0 = by * 16;
    const int n0 = blockIdx.y * BN;
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        tc::mbar_fence_init();
    }
    if (tid < 32) tc::tmem_alloc(tslot, brick_tmem_cols<BN, ZT>());
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t base = tc::saddr(tiles);
    const int nch = p.Ci / 16;
    if (tid == 0) {
        auto load = [&](int c) {
            const int s = c % S;
            const uint32_t st = base + (uint32_t)s * ST;
            tc::mbar_expect_tx(&full[s], kBytes);
            for (int h = 0; h < 2; ++h) {
                tc::tma_load_5d(st + (uint32_t)h * kPlane, &bp.tx, &full[s], 16 * c + 8 * h, x0 - 1, y0 - 1, z0 - 1, b);
                tc::tma_load_3d(st + AB + (uint32_t)h * WP, &bp.tw, &full[s], 16 * c + 8 * h, n0, 0);
            }
        };
        bool ok = true;
        int loaded = 0, issued = 0;
        for (; loaded < S && loaded < nch; ++loaded) load(loaded);
        for (int c = 0; c < nch && ok; ++c) {
            const int s = c % S;
            ok = tc::mbar_wait(&full[s], (unsigned)(c / S) & 1u, kSpin);
            if (!ok) break;
            tc::fence_after();
            const uint32_t st = base + (uint32_t)s * ST;
#pragma unroll 1
            for (int t = 0; t < 27; ++t) {
                const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
                const uint64_t bd = sdesc_lbo_sbo(st + AB + (uint32_t)t * (BN * 16u), WP, 128u);
#pragma unroll
                for (int zz = 0; zz < ZT; ++zz) {   // plane z0 + zz into accumulator columns zz BN ..
                    const uint32_t a = st + (uint32_t)((((1 + zz + dz) * kBY + 1 + dy) * kBX + 1 + dx) * 16);
                    tc::mma_bf16(tmem + (uint32_t)(zz * BN), sdesc_lbo_sbo(a, kPlane, kBX * 16u), bd, idesc,
                                 (c > 0 || t > 0) ? 1u : 0u);
                }
            }
            tc::mma_commit(&empty[s]);
            issued = c + 1;
            if (loaded < nch) {   // refill this stage once its MMAs are done
                ok = tc::mbar_wait(&empty[s], (unsigned)(c / S) & 1u, kSpin);
                if (ok) load(loaded++);
            }
        }
        // every TMA load issued must have landed before the CTA may exit
        for (int c = issued; c < loaded; ++c) tc::mbar_wait(&full[c % S], (unsigned)(c / S) & 1u, kSpin);
        s_state[0] = issued;
        s_state[1] = ok && issued == nch;
    }
    __syncthreads();
    bool ok = s_state[1] != 0;
    if (s_state[0] > 0) {
        const int c = s_state[0] - 1;
        ok = tc::mbar_wait(&empty[c % S], (unsigned)(c / S) & 1u, kSpin) && ok;
    }
    tc::fence_after();
    ok = !__syncthreads_or(!ok);
    if (!ok) {
        if (tid == 0) atomicOr(p.err, 1);
    } else {
        // row tid: x = x0 + tid % 8, y = y0 + tid / 8, at z0 .. z0 + ZT - 1
#pragma unroll 1
        for (int zz = 0; zz < ZT && z0 + zz < p.Z; ++zz) {
            const long v = (((long)b * p.Z + z0 + zz) * p.Y + y0 + tid / 8) * p.X + x0 + (tid & 7);
#pragma unroll 1
            for (int c0 = 0; c0 < BN; c0 += 16) {
                float r[16];
                tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(zz * BN + c0), r);
                store_row16(p, v, n0 + c0, r);
            }
        }
    }
    tc::fence_before();
    __syncthreads();
    if (tid < 32) {
        tc::fence_after();
        tc::tmem_free(tmem, brick_tmem_cols<BN, ZT>());
    }
}

// Operands of the weight gradient in 8-voxel groups: for a [voxel][C] tensor, group g holds the 8
// voxels 8g .. 8g+7 of every channel as C records of 16 bytes, [g][c][8].  X is a multiple of 8, so
// a group lies in one x-row and a tap's shift by (dz, dy) moves whole groups; the shift by dx is
// in the three copies of the input.
struct WgradP {
    const __nv_bfloat16 *dyt;   // [nvox/8][Co][8]  upstream gradient (after the ReLU mask)
    const __nv_bfloat16 *xs;    // [3][nvox/8][Ci][8]  layer input shifted by dx = -1, 0, +1
    float *part;                // [voxel chunk][Co][ldw], column tap * Ci + i: one partial sum per chunk
    long nvox;                  // a multiple of 8
    int Z, Y, X, Ci, Co, ntap, ldw, vchunk;   // X, Ci multiples of 8, vchunk a multiple of 16
    int *err;
};

// partial dW[o][tap, i] = sum over this CTA's voxel chunk of X[v + off(tap)][i] dY[v][o]:
// M = 128 (tap, i) rows, N = the output channels (BN >= Co), K = voxels.  Each thread copies the
// 16-byte records of its row (tap, i), one per 8-voxel group; the records of consecutive rows of a
// tap are consecutive in memory, so a warp's copies of one group cover a few contiguous runs.
// k_wsum adds the chunks' partials in chunk order, so the gradient does not depend on the order the
// CTAs finish in.
template <int BN>
__global__ void __launch_bounds__(128) k_wgrad(WgradP p) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *tiles = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *bar = reinterpret_cast<uint64_t *>(tiles + kStages * stage_bytes<BN>());
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + kStages);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int m0 = blockIdx.x * 128;
    const long vbase = (long)blockIdx.y * p.vchunk;
    const long vend = (vbase + p.vchunk < p.nvox) ? vbase + p.vchunk : p.nvox;
    const int nch = (int)((vend - vbase + 15) / 16);
    const int N = p.ntap * p.Ci;
    const long YX = (long)p.Y * p.X;
    // this thread's A row: (tap, i) = m0 + tid
    const int ng = m0 + tid;
    const bool rok = ng < N;
    int tap = 0, ci = 0, dz = 0, dy = 0, dx = 0;
    if (rok) {
        tap = ng / p.Ci;
        ci = ng - tap * p.Ci;
        if (p.ntap == 27) { dz = tap / 9 - 1; dy = (tap / 3) % 3 - 1; dx = tap % 3 - 1; }
    }
    // record of group 0 of this row's shifted input; group g's record is Ci * 8 elements further on
    const long G = p.nvox / 8, gstride = (long)p.Ci * 8;
    const __nv_bfloat16 *xrow = p.xs + ((long)(dx + 1) * G * p.Ci + ci) * 8 + (dz * YX + (long)dy * p.X) / 8 * gstride;
    const uint32_t tmem = prologue<BN>(bar, tslot);
    // (x, y, z) of voxel vbase + 16 nextc, the first voxel of the next sub-chunk to load: the main
    // loop loads the sub-chunks in increasing order, so the coordinates advance by 16 voxels per
    // load instead of being divided out of the voxel index each time (X is a multiple of 8, so an
    // 8-voxel half never leaves its x-row)
    int xq, yq, zq, nextc = 0;
    {
        const long row = vbase / p.X;
        xq = (int)(vbase - row * p.X);
        yq = (int)(row % p.Y);
        zq = (int)((row / p.Y) % p.Z);
    }
    auto next_row = [&](int &y, int &z) {
        if (++y == p.Y) {
            y = 0;
            if (++z == p.Z) z = 0;
        }
    };
    // this thread's records of the next sub-chunk's first group (A row, and B row o = tid / 2 of
    // half tid % 2 for the threads that load B), advanced with the coordinates
    const int ngroups = (int)((vend - vbase) >> 3);
    const __nv_bfloat16 *acur = xrow + (vbase >> 3) * gstride;
    constexpr int NB = (2 * BN + 127) / 128;      // B copies per thread and sub-chunk
    const __nv_bfloat16 *bcur[NB];
    uint32_t b_off[NB];
    int bh[NB];
    bool bload[NB];
#pragma unroll
    for (int r = 0; r < NB; ++r) {                // B entry i = tid + 128 r: row o = i / 2, half i % 2
        const int i = tid + 128 * r, o = i >> 1;
        bh[r] = i & 1;
        bload[r] = i < 2 * BN && o < p.Co;
        bcur[r] = p.dyt + (((vbase >> 3) + bh[r]) * p.Co + (o < p.Co ? o : 0)) * 8;
        b_off[r] = tc::tile_off(o, bh[r]);
    }
    const uint32_t a_off0 = tc::tile_off(tid, 0), a_off1 = tc::tile_off(tid, 1);
    auto load = [&](int c, uint32_t a_s, uint32_t b_s) {
        for (; nextc < c; ++nextc) {
            xq += 16;
            while (xq >= p.X) {
                xq -= p.X;
                next_row(yq, zq);
            }
            acur += 2 * gstride;
#pragma unroll
            for (int r = 0; r < NB; ++r) bcur[r] += 16 * p.Co;
        }
        const int g = 2 * c;            // the sub-chunk's first group within the chunk
        // A: row (tap, i), groups g and g + 1 (each one x-row)
        bool ok = rok && g < ngroups && (unsigned)(zq + dz) < (unsigned)p.Z && (unsigned)(yq + dy) < (unsigned)p.Y;
        tc::cp16(a_s + a_off0, ok ? acur : p.xs, ok);
        int y = yq, zz = zq;
        if (xq + 8 >= p.X) next_row(y, zz);
        ok = rok && g + 1 < ngroups && (unsigned)(zz + dz) < (unsigned)p.Z && (unsigned)(y + dy) < (unsigned)p.Y;
        tc::cp16(a_s + a_off1, ok ? acur + gstride : p.xs, ok);
        // B: row o, group g + half
#pragma unroll
        for (int r = 0; r < NB; ++r)
            if (tid + 128 * r < 2 * BN) {
                const bool okb = bload[r] && g + bh[r] < ngroups;
                tc::cp16(b_s + b_off[r], okb ? bcur[r] : p.dyt, okb);
            }
    };
    int issued;
    const bool ok = mainloop<BN>(load, nch, tiles, bar, tmem, &issued);
    if (!ok) {
        if (tid == 0) atomicOr(p.err, 1);
    } else {
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 16) {
            float r[16];
            tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
            if (!rok) continue;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int o = c0 + j;
                if (o < p.Co) p.part[((long)blockIdx.y * p.Co + o) * p.ldw + ng] = r[j];
            }
        }
    }
    epilogue_free<BN>(tmem);
}

// dw[o][col] += sum over chunks s = 0, 1, ... of part[s][o][col], for the N real columns
__global__ void k_wsum(float *__restrict__ dw, const float *__restrict__ part, int nchunk, int Co, int N, int ldw) {
    const long n = (long)Co * N;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const int o = (int)(i / N), col = (int)(i - (long)o * N);
        const long e = (long)o * ldw + col;
        float s = 0.f;
        for (int c = 0; c < nchunk; ++c) s += part[(long)c * Co * ldw + e];
        dw[e] += s;
    }
}

// db[c] += sum over blocks b = 0, 1, ... of part[b][c]: one block per channel, a fixed strided
// sum per thread and a fixed tree over the threads (independent of scheduling)
__global__ void __launch_bounds__(256) k_colsum(float *__restrict__ db, const float *__restrict__ part, long nb, int C) {
    __shared__ float red[256];
    const int c = blockIdx.x;
    float s = 0.f;
    for (long b = threadIdx.x; b < nb; b += 256) s += part[b * C + c];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) db[c] += red[0];
}

// ---- memory-bound helpers ---------------------------------------------------------------------

// [B][C][Z][Y][X] float -> [voxel][Cp] BF16 (channels C..Cp-1 zero)
__global__ void k_to_ndhwc(const float *__restrict__ in, __nv_bfloat16 *__restrict__ out, long V, int C, int Cp, long vps) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < V * Cp; i += (long)gridDim.x * blockDim.x) {
        const long v = i / Cp;
        const int c = (int)(i - v * Cp);
        const long b = v / vps, s = v - b * vps;
        out[i] = __float2bfloat16_rn(c < C ? in[(b * C + c) * vps + s] : 0.f);
    }
}
// [B][C][Z][Y][X] float -> [voxel][Cp] float (channels C..Cp-1 zero)
__global__ void k_to_ndhwc_f32(const float *__restrict__ in, float *__restrict__ out, long V, int C, int Cp, long vps) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < V * Cp; i += (long)gridDim.x * blockDim.x) {
        const long v = i / Cp;
        const int c = (int)(i - v * Cp);
        const long b = v / vps, s = v - b * vps;
        out[i] = c < C ? in[(b * C + c) * vps + s] : 0.f;
    }
}
// first C channels of [voxel][Cp] float -> [B][C][Z][Y][X] float
__global__ void k_from_ndhwc_f32(const float *__restrict__ in, float *__restrict__ out, long V, int C, int Cp, long vps) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < V * C; i += (long)gridDim.x * blockDim.x) {
        const long b = i / (C * vps), r = i - b * C * vps;
        const int c = (int)(r / vps);
        const long s = r - (long)c * vps;
        out[i] = in[(b * vps + s) * Cp + c];
    }
}

// 2x2x2 average pooling, BF16 [voxel][C] at (Z, Y, X) -> half resolution
__global__ void k_pool(const __nv_bfloat16 *__restrict__ in, __nv_bfloat16 *__restrict__ out, long Vh, int C, int Zh,
                       int Yh, int Xh) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < Vh * C; i += (long)gridDim.x * blockDim.x) {
        const long vh = i / C;
        const int c = (int)(i - vh * C);
        long q = vh;
        const int x = (int)(q % Xh); q /= Xh;
        const int y = (int)(q % Yh); q /= Yh;
        const int z = (int)(q % Zh);
        const long b = q / Zh;
        float s = 0.f;
        for (int d = 0; d < 8; ++d) {
            const long v = (((b * 2 * Zh + 2 * z + (d >> 2)) * 2 * Yh + 2 * y + ((d >> 1) & 1)) * 2 * Xh + 2 * x + (d & 1));
            s += __bfloat162float(in[v * C + c]);
        }
        out[i] = __float2bfloat16_rn(0.125f * s);
    }
}
// gradient of k_pool: out[v][c] (+)= g[parent(v)][c] / 8   (float)
__global__ void k_pool_bwd(const float *__restrict__ g, float *__restrict__ out, long V, int C, int Z, int Y, int X,
                           int accumulate) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < V * C; i += (long)gridDim.x * blockDim.x) {
        const long v = i / C;
        const int c = (int)(i - v * C);
        long q = v;
        const int x = (int)(q % X); q /= X;
        const int y = (int)(q % Y); q /= Y;
        const int z = (int)(q % Z);
        const long b = q / Z;
        const long vh = ((b * (Z / 2) + z / 2) * (Y / 2) + y / 2) * (X / 2) + x / 2;
        const float a = 0.125f * g[vh * C + c];
        out[i] = accumulate ? out[i] + a : a;
    }
}
// nearest upsampling of deep [voxel/8][Cd] concatenated with skip [voxel][Cs] -> [voxel][Cd + Cs]
__global__ void k_upcat(const __nv_bfloat16 *__restrict__ deep, const __nv_bfloat16 *__restrict__ skip,
                        __nv_bfloat16 *__restrict__ out, long V, int Cd, int Cs, int Z, int Y, int X) {
    const int C = Cd + Cs;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < V * C; i += (long)gridDim.x * blockDim.x) {
        const long v = i / C;
        const int c = (int)(i - v * C);
        if (c >= Cd) {
            out[i] = skip[v * Cs + (c - Cd)];
            continue;
        }
        long q = v;
        const int x = (int)(q % X); q /= X;
        const int y = (int)(q % Y); q /= Y;
        const int z = (int)(q % Z);
        const long b = q / Z;
        const long vh = ((b * (Z / 2) + z / 2) * (Y / 2) + y / 2) * (X / 2) + x / 2;
        out[i] = deep[vh * Cd + c];
    }
}
// gradient of k_upcat: deep gradient (sum over the 8 children) and skip gradient (copy)
__global__ void k_upcat_bwd(const float *__restrict__ g, float *__restrict__ gdeep, float *__restrict__ gskip, long Vh,
                            int Cd, int Cs, int Zh, int Yh, int Xh) {
    const int C = Cd + Cs;
    const long V = Vh * 8;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < Vh * Cd + V * Cs; i += (long)gridDim.x * blockDim.x) {
        if (i >= Vh * Cd) {
            const long j = i - Vh * Cd, v = j / Cs;
            const int c = (int)(j - v * Cs);
            gskip[j] = g[v * C + Cd + c];
            continue;
        }
        const long vh = i / Cd;
        const int c = (int)(i - vh * Cd);
        long q = vh;
        const int x = (int)(q % Xh); q /= Xh;
        const int y = (int)(q % Yh); q /= Yh;
        const int z = (int)(q % Zh);
        const long b = q / Zh;
        float s = 0.f;
        for (int d = 0; d < 8; ++d) {
            const long v = (((b * 2 * Zh + 2 * z + (d >> 2)) * 2 * Yh + 2 * y + ((d >> 1) & 1)) * 2 * Xh + 2 * x + (d & 1));
            s += g[v * C + c];
        }
        gdeep[i] = s;
    }
}

// ReLU backward and the operands of the layer's backward GEMMs:
//   d[v][c] = g[v][c] * (out[v][c] > 0)  (out null: no ReLU)  -> BF16 [voxel][C] and, in 8-voxel
//   groups for the weight gradient, dt [V/8][C][8] (V a multiple of 8),
//   dbp[block][c] = sum over the block's 32 voxels of d[v][c] (k_colsum adds the blocks in order).
//   Block: 32 voxels x C channels through shared memory.
__global__ void k_relu_bwd(const float *__restrict__ g, const __nv_bfloat16 *__restrict__ out,
                           __nv_bfloat16 *__restrict__ d, __nv_bfloat16 *__restrict__ dt, float *__restrict__ dbp, long V,
                           int C) {
    __shared__ float tile[32][129];
    const long v0 = (long)blockIdx.x * 32;
    for (int i = threadIdx.x; i < 32 * C; i += blockDim.x) {
        const int r = i / C, c = i - r * C;
        const long v = v0 + r;
        float a = 0.f;
        if (v < V) {
            a = g[v * C + c];
            if (out && !(__bfloat162float(out[v * C + c]) > 0.f)) a = 0.f;
            d[v * C + c] = __float2bfloat16_rn(a);
        }
        tile[r][c] = __bfloat162float(__float2bfloat16_rn(a));
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 32 * C; i += blockDim.x) {
        const int c = i / 32, r = i - c * 32;
        const long v = v0 + r;
        if (v < V) dt[((v >> 3) * C + c) * 8 + (v & 7)] = __float2bfloat16_rn(tile[r][c]);
    }
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        float s = 0.f;
        for (int r = 0; r < 32; ++r) s += tile[r][c];
        dbp[(long)blockIdx.x * C + c] = s;
    }
}

// k_relu_bwd for C a multiple of 8 and 16-byte aligned buffers: a block takes VB voxels (a multiple
// of 16, VB C <= 8192), reads g and out with 16- and 8-byte loads, writes d with 8-byte stores and
// dt as pairs of 16-byte channel records of 8 voxels, and leaves one per-channel partial sum of the
// block's (BF16-rounded) gradient in dbp; same values as k_relu_bwd, partial sums over VB voxels.
__global__ void __launch_bounds__(256) k_relu_bwd_v(const float *__restrict__ g, const __nv_bfloat16 *__restrict__ out,
                                                    __nv_bfloat16 *__restrict__ d, __nv_bfloat16 *__restrict__ dt,
                                                    float *__restrict__ dbp, long V, int C, int VB) {
    extern __shared__ float rtile[];                 // [VB][C + 1]
    const int ld = C + 1;
    const long v0 = (long)blockIdx.x * VB;
    const int n4 = VB * C / 4;
    for (int i = threadIdx.x; i < n4; i += blockDim.x) {
        const int e = 4 * i, r = e / C, c = e - r * C;
        const long v = v0 + r;
        float a[4] = {0.f, 0.f, 0.f, 0.f};
        if (v < V) {
            const float4 q = reinterpret_cast<const float4 *>(g + v * C + c)[0];
            a[0] = q.x; a[1] = q.y; a[2] = q.z; a[3] = q.w;
            if (out) {
                alignas(8) __nv_bfloat16 o[4];
                *reinterpret_cast<uint2 *>(o) = *reinterpret_cast<const uint2 *>(out + v * C + c);
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (!(__bfloat162float(o[k]) > 0.f)) a[k] = 0.f;
            }
            alignas(8) __nv_bfloat16 b[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) b[k] = __float2bfloat16_rn(a[k]);
            *reinterpret_cast<uint2 *>(d + v * C + c) = *reinterpret_cast<const uint2 *>(b);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) rtile[r * ld + c + k] = __bfloat162float(__float2bfloat16_rn(a[k]));
    }
    __syncthreads();
    const int ng = VB / 16;
    for (int w = threadIdx.x; w < C * ng; w += blockDim.x) {
        const int c = w % C, gq = w / C;                 // consecutive threads: consecutive records
        const long vs = v0 + 16L * gq;
        if (vs >= V) continue;
        alignas(16) __nv_bfloat16 val[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) val[k] = __float2bfloat16_rn(rtile[(16 * gq + k) * ld + c]);
        uint4 *dst = reinterpret_cast<uint4 *>(dt + ((vs >> 3) * C + c) * 8);
        dst[0] = reinterpret_cast<const uint4 *>(val)[0];
        if (vs + 16 <= V) dst[C] = reinterpret_cast<const uint4 *>(val)[1];
    }
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        float sum = 0.f;
        for (int r = 0; r < VB; ++r) sum += rtile[r * ld + c];
        dbp[(long)blockIdx.x * C + c] = sum;
    }
}
inline int relu_bwd_vb(int C) {
    int vb = 8192 / C;
    vb = vb > 256 ? 256 : (vb < 16 ? 16 : vb);
    return vb / 16 * 16;
}
inline size_t relu_bwd_smem(int C) { return (size_t)relu_bwd_vb(C) * (C + 1) * sizeof(float); }

// k_upcat for Cd and Cs multiples of 8 and 16-byte aligned buffers: one 16-byte group of 8 channels
// per thread and step (each group lies wholly in the deep or the skip part)
__global__ void k_upcat_v(const __nv_bfloat16 *__restrict__ deep, const __nv_bfloat16 *__restrict__ skip,
                          __nv_bfloat16 *__restrict__ out, long V, int Cd, int Cs, int Z, int Y, int X) {
    const int Cdg = Cd / 8, Csg = Cs / 8, Cg = Cdg + Csg;
    const uint4 *dp = reinterpret_cast<const uint4 *>(deep), *sp = reinterpret_cast<const uint4 *>(skip);
    uint4 *op = reinterpret_cast<uint4 *>(out);
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < V * Cg; i += (long)gridDim.x * blockDim.x) {
        const long v = i / Cg;
        const int gq = (int)(i - v * Cg);
        if (gq >= Cdg) {
            op[i] = sp[v * Csg + (gq - Cdg)];
            continue;
        }
        long q = v;
        const int x = (int)(q % X); q /= X;
        const int y = (int)(q % Y); q /= Y;
        const int z = (int)(q % Z);
        const long b = q / Z;
        const long vh = ((b * (Z / 2) + z / 2) * (Y / 2) + y / 2) * (X / 2) + x / 2;
        op[i] = dp[vh * Cdg + gq];
    }
}

// x [V][C] (channels last, BF16) -> xs [j][V/8][C][8] with xs[j][g][c][k] = x[8g + k + j - 1][c]
// when the x coordinate of voxel 8g + k plus j - 1 stays in [0, X), else 0 (j = 0, 1, 2; nshift = 1
// writes j = 1 only): the weight gradient's input in 8-voxel groups (k_wgrad), in three copies
// shifted along x so that a tap's shift along x needs no realignment.  A block takes VB voxels (a
// multiple of 16, (VB + 2) C elements of shared memory): the input around them is one contiguous
// range, copied with 16-byte loads; each thread then assembles 16 consecutive voxels of one (j, c)
// row and writes them as two 16-byte channel records.  C, X and V are multiples of 8 (the
// network's shapes).
__global__ void __launch_bounds__(256) k_xshift(const __nv_bfloat16 *__restrict__ x, __nv_bfloat16 *__restrict__ xs,
                                                long V, int C, int X, int nshift, int VB) {
    extern __shared__ uint4 xsm[];
    const __nv_bfloat16 *tile = reinterpret_cast<const __nv_bfloat16 *>(xsm);   // [VB + 2][C], row r = voxel v0 - 1 + r
    const long v0 = (long)blockIdx.x * VB;
    const int cq = C / 8;                                   // 16-byte pieces per voxel
    const int n16 = (VB + 2) * cq;
    const uint4 *src = reinterpret_cast<const uint4 *>(x);
    for (int i = threadIdx.x; i < n16; i += blockDim.x) {
        const long v = v0 - 1 + i / cq;
        xsm[i] = (v >= 0 && v < V) ? src[(v0 - 1) * cq + i] : make_uint4(0u, 0u, 0u, 0u);
    }
    __syncthreads();
    const int j0 = nshift == 3 ? 0 : 1;
    const int ng = VB / 16;
    for (int w = threadIdx.x; w < nshift * C * ng; w += blockDim.x) {
        const int c = w % C, rest = w / C;
        const int g = rest % ng, j = j0 + rest / ng;
        const long vs = v0 + 16L * g;                       // first voxel of this run
        if (vs >= V) continue;
        alignas(16) __nv_bfloat16 val[16];
        int xv = (int)(vs % X);                             // x coordinate of voxel vs + k
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const bool in = vs + k < V && (unsigned)(xv + j - 1) < (unsigned)X;
            val[k] = in ? tile[(16 * g + k + j) * C + c] : __float2bfloat16_rn(0.f);
            if (++xv == X) xv = 0;
        }
        // groups vs / 8 and vs / 8 + 1 (the second one only inside the tensor: V is a multiple of 8)
        uint4 *dst = reinterpret_cast<uint4 *>(xs + (((long)j * (V / 8) + vs / 8) * C + c) * 8);
        dst[0] = reinterpret_cast<const uint4 *>(val)[0];
        if (vs + 16 <= V) dst[C] = reinterpret_cast<const uint4 *>(val)[1];
    }
}
// voxels per block of k_xshift for C channels, and its shared memory
inline int xshift_vb(int C) {
    int vb = 8192 / C;
    vb = vb > 256 ? 256 : (vb < 16 ? 16 : vb);
    return vb / 16 * 16;
}
inline size_t xshift_smem(int C) { return (size_t)(xshift_vb(C) + 2) * C * sizeof(__nv_bfloat16); }

// squared error of y [n] against t divided by denom (the number of real elements; padded channels
// hold 0 in both), one partial sum per block (k_dsum adds them in order), and its gradient
// 2 (y - t) / denom as FP32
__global__ void k_mse(const float *__restrict__ y, const float *__restrict__ t, float *__restrict__ g, long n,
                      double denom, double *__restrict__ part) {
    __shared__ double red[32];
    double s = 0.0;
    const float sc = (float)(2.0 / denom);
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const float d = y[i] - t[i];
        s += (double)d * d;
        g[i] = sc * d;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a += red[w];
        part[blockIdx.x] = a / denom;
    }
}

// loss = sum over blocks b = 0, 1, ... of part[b] (one block of 256 threads, fixed order)
__global__ void __launch_bounds__(256) k_dsum(double *__restrict__ loss, const double *__restrict__ part, int nb) {
    __shared__ double red[256];
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += 256) s += part[b];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = red[0];
}

__global__ void k_add(float *__restrict__ a, const float *__restrict__ b, long n) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) a[i] += b[i];
}

// Adam on one layer (master weights [Co][Kp] FP32 in the GEMM layout, bias [Co]); refreshes the
// BF16 forward weights and the BF16 transposed weights of the data-gradient convolution:
//     wt[i][tap' * Co + o] = w[o][(ntap - 1 - tap') * Ci + i]
struct AdamP {
    float *w, *m, *v, *gw;        // [Co][Kp]
    float *b, *mb, *vb, *gb;      // [Co]
    __nv_bfloat16 *wf, *wt;       // forward [Co][Kp], transposed [Ci][Kpt] (may be null)
    __nv_bfloat16 *wfb, *wtb;     // brick-kernel copies [27][Co][Ci] and [27][Ci][Co] (3x3x3 only)
    int Co, Ci, ntap, Kp, Kpt;
    float lr, b1, b2, eps, c1, c2;   // c1 = 1 - b1^k, c2 = 1 - b2^k
};
__global__ void k_adam(AdamP p) {
    const long nw = (long)p.Co * p.Kp;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < nw + p.Co; i += (long)gridDim.x * blockDim.x) {
        float *w, *m, *v, g;
        if (i < nw) { w = p.w + i; m = p.m + i; v = p.v + i; g = p.gw[i]; }
        else { const long j = i - nw; w = p.b + j; m = p.mb + j; v = p.vb + j; g = p.gb[j]; }
        const float mm = p.b1 * *m + (1.f - p.b1) * g;
        const float vv = p.b2 * *v + (1.f - p.b2) * g * g;
        *m = mm;
        *v = vv;
        const float nw_ = *w - p.lr * (mm / p.c1) / (sqrtf(vv / p.c2) + p.eps);
        *w = nw_;
        if (i < nw) {
            p.wf[i] = __float2bfloat16_rn(nw_);
            const int o = (int)(i / p.Kp), k = (int)(i - (long)o * p.Kp);
            if (k < p.ntap * p.Ci) {
                const int tap = k / p.Ci, ci = k - tap * p.Ci;
                const __nv_bfloat16 h = __float2bfloat16_rn(nw_);
                if (p.wt) p.wt[(long)ci * p.Kpt + (p.ntap - 1 - tap) * p.Co + o] = h;
                if (p.wfb) p.wfb[((long)tap * p.Co + o) * p.Ci + ci] = h;
                if (p.wtb) p.wtb[((long)(p.ntap - 1 - tap) * p.Ci + ci) * p.Co + o] = h;
            }
        }
    }
}

// BF16 copies of master weights (after a host upload): forward and transposed layouts
__global__ void k_wcopy(const float *__restrict__ w, __nv_bfloat16 *__restrict__ wf, __nv_bfloat16 *__restrict__ wt,
                        __nv_bfloat16 *__restrict__ wfb, __nv_bfloat16 *__restrict__ wtb, int Co, int Ci, int ntap,
                        int Kp, int Kpt) {
    const long nw = (long)Co * Kp;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < nw; i += (long)gridDim.x * blockDim.x) {
        const float a = w[i];
        const __nv_bfloat16 h = __float2bfloat16_rn(a);
        wf[i] = h;
        const int o = (int)(i / Kp), k = (int)(i - (long)o * Kp);
        if (k < ntap * Ci) {
            const int tap = k / Ci, ci = k - tap * Ci;
            if (wt) wt[(long)ci * Kpt + (ntap - 1 - tap) * Co + o] = h;
            if (wfb) wfb[((long)tap * Co + o) * Ci + ci] = h;
            if (wtb) wtb[((long)(ntap - 1 - tap) * Ci + ci) * Co + o] = h;
        }
    }
}

// He-normal initialisation of one layer's master weights [Co][Kp] (zero in the padding columns):
// standard normals by the Box-Muller transform of two Philox4x32-10 outputs keyed by the seed,
// counters (layer, element, 0 / 1)
__global__ void k_init_he(float *__restrict__ w, int Co, int Kp, int K, float sd, uint32_t layer, uint32_t k0,
                          uint32_t k1) {
    const long n = (long)Co * Kp;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const int k = (int)(i % Kp);
        if (k >= K) { w[i] = 0.f; continue; }
        const uint32_t u1 = philox_first(layer, (uint32_t)i, 0u, 0u, k0, k1);
        const uint32_t u2 = philox_first(layer, (uint32_t)i, 1u, 0u, k0, k1);
        const double a = ((double)u1 + 0.5) * 2.3283064365386963e-10, b = ((double)u2 + 0.5) * 2.3283064365386963e-10;
        w[i] = (float)(sd * sqrt(-2.0 * log(a)) * cos(6.283185307179586 * b));
    }
}

}  // namespace unet
}  // namespace tdgl
