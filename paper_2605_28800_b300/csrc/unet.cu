// libtdgl: the learned warm start (tdgl_unet_* and tdgl_conv3d* of include/tdgl.h).
//
// A 3D U-Net whose convolutions run on the tensor cores (unet_kernels.cuh).  The host side owns
// the layer table, the device buffers of one batch of activations and gradients, the FP32 master
// weights with their Adam moments, and issues every launch on the context's stream.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "runtime.cuh"
#include "unet_kernels.cuh"

using namespace tdgl;
using namespace tdgl::unet;
using namespace tdgl_rt;

namespace {

int pad16(int k) { return (k + 15) & ~15; }
int grid_n(long n) { return (int)std::min<long>(std::max<long>((n + 255) / 256, 1), 148L * 32); }

struct Dims {
    int Z, Y, X;
    long vps() const { return (long)Z * Y * X; }
};

// one convolution
struct Layer {
    int Ci, Co, ntap, Kp, Kpt;      // Kp = pad16(ntap Ci), Kpt = pad16(ntap Co)
    int ci_real, co_real;           // channels at the boundary (layer 0 input and the head
                                    // output are padded to 8 inside)
    int lev;                        // resolution level
    bool relu, need_dx;
    size_t ow, ob;                  // offsets of w [Co][Kp] and b [Co] in the parameter arrays
    __nv_bfloat16 *wf = nullptr, *wt = nullptr;
    __nv_bfloat16 *wfb = nullptr, *wtb = nullptr;   // brick-kernel weights [27][Co][Ci], [27][Ci][Co]
    // activation buffers (set per network): input, output (BF16 or, for the head, FP32)
    __nv_bfloat16 *in = nullptr;
    void *out = nullptr;
    float *g_out = nullptr, *g_in = nullptr;   // gradients of output and input (FP32)
};

template <int BN>
int set_attr() {
    cudaError_t e = cudaFuncSetAttribute(k_conv<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gemm_smem<BN>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_wgrad<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gemm_smem<BN>());
    return e == cudaSuccess ? 0 : -1;
}

int conv_bn(int co) {
    for (int bn : {128, 64, 32, 16})
        if (co % bn == 0) return bn;
    return 16;
}

// activations [B][Z][Y][X][C] BF16 as (C, X, Y, Z, B), box (8, 10, 18, zt + 2, 1): one 8-channel
// plane of a brick with its halo for zt output planes; out-of-range voxels read as zero
bool act_map(CUtensorMap *m, const void *x, int C, Dims d, long B, int zt) {
    auto enc = tmap_encode();
    if (!enc) return false;
    const cuuint64_t dims[5] = {(cuuint64_t)C, (cuuint64_t)d.X, (cuuint64_t)d.Y, (cuuint64_t)d.Z, (cuuint64_t)B};
    const cuuint64_t e = 2;
    const cuuint64_t strides[4] = {C * e, (cuuint64_t)d.X * C * e, (cuuint64_t)d.Y * d.X * C * e,
                                   (cuuint64_t)d.Z * d.Y * d.X * C * e};
    const cuuint32_t box[5] = {8, (cuuint32_t)kBX, (cuuint32_t)kBY, (cuuint32_t)(zt + 2), 1};
    const cuuint32_t es[5] = {1, 1, 1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void *>(x), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// brick weights [27][Co][Ci] BF16 as (Ci, Co, 27), box (8, bn, 27): one half of a chunk, all taps
bool wgt_map(CUtensorMap *m, const void *w, int Ci, int Co, int bn) {
    auto enc = tmap_encode();
    if (!enc) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)Ci, (cuuint64_t)Co, 27};
    const cuuint64_t strides[2] = {(cuuint64_t)Ci * 2, (cuuint64_t)Co * Ci * 2};
    const cuuint32_t box[3] = {8, (cuuint32_t)bn, 27};
    const cuuint32_t es[3] = {1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(w), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Y[v][o] = act(b + conv(X, W)) over nvox voxels of dims d.  w: gather-kernel weights [Co][Kp];
// wb: the same weights as [27][Co][Ci] for the brick kernel (null: gather kernel only)
int launch_conv(tdgl_ctx *ctx, const __nv_bfloat16 *x, const __nv_bfloat16 *w, const __nv_bfloat16 *wb, const float *b,
                void *y, long nvox, Dims d, int Ci, int Co, int ntap, int Kp, bool relu, bool f32out, int *err) {
    ConvP p{x, w, b, y, nvox, d.Z, d.Y, d.X, Ci, Co, ntap, Kp / 8, relu ? 1 : 0, f32out ? 1 : 0, err, 1, nullptr};
    // the brick kernel: 3x3x3, 16-channel input chunks, 8 x 16 voxel bricks, output tiles up to 64
    if (wb && ntap == 27 && Ci % 16 == 0 && d.X % 8 == 0 && d.Y % 16 == 0) {
        const int bn = Co % 64 == 0 ? 64 : (Co % 32 == 0 ? 32 : 16);
        BrickP bp;
        memset(&bp, 0, sizeof bp);
        bp.c = p;
        const bool one = Ci == 16;
        // CTAs of 8 x 16 voxels in zt z planes: two planes while that still gives at least one CTA
        // per SM (they share one brick and one weight load), else one
        const long B = nvox / d.vps(), ntile = (Co + bn - 1) / bn;
        const int zt = (long)(d.X / 8) * (d.Y / 16) * ((d.Z + 1) / 2) * B * ntile >= ctx->nsm ? 2 : 1;
        if (!act_map(&bp.tx, x, Ci, d, B, zt) || !wgt_map(&bp.tw, wb, Ci, Co, bn))
            return fail(ctx, TDGL_ECUDA, "cannot encode the tensor maps of a convolution");
        const dim3 grid((unsigned)((long)(d.X / 8) * (d.Y / 16) * ((d.Z + zt - 1) / zt) * B), (unsigned)ntile);
        return launch(ctx, TDGL_K_UNET, [&] {
#define TDGL_BRICK(BN_, S_, ZT_) k_conv_brick<BN_, S_, ZT_><<<grid, 128, brick_smem<BN_, S_, ZT_>(), ctx->stream>>>(bp)
#define TDGL_BRICK_Z(BN_, S_) if (zt == 2) TDGL_BRICK(BN_, S_, 2); else TDGL_BRICK(BN_, S_, 1)
            switch (bn) {
                case 64: if (one) { TDGL_BRICK_Z(64, 1); } else { TDGL_BRICK_Z(64, 2); } break;
                case 32: if (one) { TDGL_BRICK_Z(32, 1); } else { TDGL_BRICK_Z(32, 2); } break;
                default: if (one) { TDGL_BRICK_Z(16, 1); } else { TDGL_BRICK_Z(16, 2); } break;
            }
#undef TDGL_BRICK_Z
#undef TDGL_BRICK
        });
    }
    const int bn = conv_bn(Co);
    dim3 grid((unsigned)((nvox + 127) / 128), (unsigned)((Co + bn - 1) / bn));
    // layers with fewer CTAs than half the SMs (the deepest levels) split their K range so that
    // about one CTA per SM works; at least four sub-chunks per split, and no split left empty
    const int nsub = p.G / 2;
    const long ctas = (long)grid.x * grid.y;
    if (2 * ctas < ctx->nsm && nsub >= 8) {
        int S = (int)std::min<long>((ctx->nsm + ctas - 1) / ctas, nsub / 4);
        const int per = (nsub + S - 1) / S;
        S = (nsub + per - 1) / per;
        if (S > 1) {
            const size_t need = (size_t)S * nvox * Co;
            if (need > ctx->splitk_n) {
                cudaFree(ctx->splitk);
                ctx->splitk = nullptr;
                ctx->splitk_n = 0;
                CK(ctx, cudaMalloc(&ctx->splitk, need * sizeof(float)));
                ctx->splitk_n = need;
            }
            p.ksplit = S;
            p.part = ctx->splitk;
            grid.z = (unsigned)S;
        }
    }
    TRY(launch(ctx, TDGL_K_UNET, [&] {
        switch (bn) {
            case 128: k_conv<128><<<grid, 128, gemm_smem<128>(), ctx->stream>>>(p); break;
            case 64: k_conv<64><<<grid, 128, gemm_smem<64>(), ctx->stream>>>(p); break;
            case 32: k_conv<32><<<grid, 128, gemm_smem<32>(), ctx->stream>>>(p); break;
            default: k_conv<16><<<grid, 128, gemm_smem<16>(), ctx->stream>>>(p); break;
        }
    }));
    if (p.ksplit == 1) return TDGL_OK;
    return launch(ctx, TDGL_K_UNET, [&] {
        k_splitk_sum<<<grid_n(nvox * Co), 256, 0, ctx->stream>>>(p.part, p.ksplit, nvox, Co, b, p.relu, p.f32out, y);
    });
}

// dW[o][tap Ci + i] += sum_v xs[dx + 1][v + dz YX + dy X][i] dY[v][o] (both operands in 8-voxel groups)
// voxels per CTA of the weight gradient (about four CTAs per SM over the (tap, i) tiles; a multiple
// of the 64 voxels of a pipeline stage) and the number of voxel chunks, each leaving one partial
// gradient
long wgrad_vchunk(long nvox, int N) {
    const long ntile = (N + 127) / 128;
    const long v = (nvox * ntile + 591) / 592;
    return std::min<long>(std::max<long>((v + 63) / 64 * 64, 256), 16384);
}
long wgrad_chunks(long nvox, int N) { return (nvox + wgrad_vchunk(nvox, N) - 1) / wgrad_vchunk(nvox, N); }
// floats of the partial-gradient workspace of one convolution (weights, then biases)
size_t wgrad_part_floats(long nvox, int Ci, int Co, int ntap, int ldw) {
    return (size_t)wgrad_chunks(nvox, ntap * Ci) * Co * ldw;
}
size_t bias_part_floats(long nvox, int Co) { return (size_t)((nvox + 31) / 32) * Co; }

// dw += the weight gradient: per-chunk partials into part, then summed in chunk order
int launch_wgrad(tdgl_ctx *ctx, const __nv_bfloat16 *dyt, const __nv_bfloat16 *xs, float *dw, float *part, long nvox,
                 Dims d, int Ci, int Co, int ntap, int ldw, int *err) {
    const int N = ntap * Ci;
    if (nvox % 8 || d.X % 8 || Ci % 8 || Co > 128)
        return fail(ctx, TDGL_EINVAL, "weight gradient: voxels, x extent and input channels multiples of 8, at most 128 outputs");
    const int bn = Co <= 16 ? 16 : (Co <= 32 ? 32 : (Co <= 64 ? 64 : 128));
    const long ntile = (N + 127) / 128;
    const long vchunk = wgrad_vchunk(nvox, N), nchunk = wgrad_chunks(nvox, N);
    WgradP p{dyt, xs, part, nvox, d.Z, d.Y, d.X, Ci, Co, ntap, ldw, (int)vchunk, err};
    const dim3 grid((unsigned)ntile, (unsigned)nchunk);
    TRY(launch(ctx, TDGL_K_UNET, [&] {
        switch (bn) {
            case 128: k_wgrad<128><<<grid, 128, gemm_smem<128>(), ctx->stream>>>(p); break;
            case 64: k_wgrad<64><<<grid, 128, gemm_smem<64>(), ctx->stream>>>(p); break;
            case 32: k_wgrad<32><<<grid, 128, gemm_smem<32>(), ctx->stream>>>(p); break;
            default: k_wgrad<16><<<grid, 128, gemm_smem<16>(), ctx->stream>>>(p); break;
        }
    }));
    return launch(ctx, TDGL_K_UNET, [&] {
        k_wsum<<<grid_n((long)Co * N), 256, 0, ctx->stream>>>(dw, part, (int)nchunk, Co, N, ldw);
    });
}

// ReLU mask of the upstream gradient (BF16, [voxel][C] and in 8-voxel groups) and db += its sum over voxels:
// per-block partials into part, summed in block order
bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

int launch_relu_bwd(tdgl_ctx *ctx, const float *g, const __nv_bfloat16 *out, __nv_bfloat16 *d, __nv_bfloat16 *dt,
                    float *db, float *part, long V, int C) {
    // the vector form for 8-channel groups and aligned buffers (the network's), else 32 voxels per block
    const bool vec = C % 8 == 0 && V % 8 == 0 && aligned16(g) && aligned16(d) && aligned16(dt) && (!out || aligned16(out));
    const int vb = vec ? relu_bwd_vb(C) : 32;
    const long nb = (V + vb - 1) / vb;      // <= (V + 31) / 32: the partial buffer's size
    TRY(launch(ctx, TDGL_K_UNET, [&] {
        if (vec) k_relu_bwd_v<<<(unsigned)nb, 256, relu_bwd_smem(C), ctx->stream>>>(g, out, d, dt, part, V, C, vb);
        else k_relu_bwd<<<(unsigned)nb, 256, 0, ctx->stream>>>(g, out, d, dt, part, V, C);
    }));
    return launch(ctx, TDGL_K_UNET, [&] { k_colsum<<<(unsigned)C, 256, 0, ctx->stream>>>(db, part, nb, C); });
}

template <int BN, int S>
int set_brick_attr() {
    return cudaFuncSetAttribute(k_conv_brick<BN, S, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)brick_smem<BN, S, 1>()) == cudaSuccess &&
                   cudaFuncSetAttribute(k_conv_brick<BN, S, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)brick_smem<BN, S, 2>()) == cudaSuccess
               ? 0
               : -1;
}

int init_attrs(tdgl_ctx *ctx) {
    if (set_attr<128>() || set_attr<64>() || set_attr<32>() || set_attr<16>() || set_brick_attr<64, 1>() ||
        set_brick_attr<64, 2>() || set_brick_attr<32, 1>() || set_brick_attr<32, 2>() || set_brick_attr<16, 1>() ||
        set_brick_attr<16, 2>())
        return fail(ctx, TDGL_ECUDA, "cannot raise the shared-memory limit of the tensor-core kernels");
    return TDGL_OK;
}

int check_err(tdgl_ctx *ctx, int *derr) {
    int h = 0;
    CK(ctx, cudaMemcpyAsync(&h, derr, sizeof h, cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    if (h) {
        cudaMemsetAsync(derr, 0, sizeof(int), ctx->stream);
        return fail(ctx, TDGL_ETIMEOUT, "tensor-core pipeline wait timed out");
    }
    return TDGL_OK;
}

}  // namespace

struct tdgl_unet {
    tdgl_ctx *ctx = nullptr;
    int cin = 0, cout = 0, coutp = 8, levels = 0, maxb = 0;   // coutp: head channels padded to 8
    int chans[8] = {0};
    Dims dims[8];
    std::vector<Layer> L;               // encoder (2 per level), decoder (2 per level), head
    size_t nparam = 0;                  // floats in the GEMM layout (w [Co][Kp] + b per layer)
    long nflat = 0;                     // floats of the boundary parameter vector
    float *P = nullptr, *G = nullptr, *M = nullptr, *V = nullptr;
    long step = 0;
    std::vector<void *> bufs;           // every device allocation, freed on destroy
    __nv_bfloat16 *xin = nullptr;       // [V0][8]
    float *tgt = nullptr, *yout = nullptr;   // [V0][coutp]
    __nv_bfloat16 *dpre = nullptr, *dpret = nullptr, *xs = nullptr;   // backward scratch
    float *wpart = nullptr, *bpart = nullptr;                          // partial gradients
    double *dloss = nullptr, *lpart = nullptr;   // loss and its per-block partials
    int *derr = nullptr;
    float *hx = nullptr, *hy = nullptr;  // device staging of host tensors
};

namespace {

template <class T>
int dalloc(tdgl_unet *n, T **p, size_t count) {
    void *q = nullptr;
    CK(n->ctx, cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T)));
    CK(n->ctx, cudaMemsetAsync(q, 0, std::max<size_t>(count, 1) * sizeof(T), n->ctx->stream));
    n->bufs.push_back(q);
    *p = reinterpret_cast<T *>(q);
    return TDGL_OK;
}

long nvox(const tdgl_unet *n, int lev, int B) { return (long)B * n->dims[lev].vps(); }

int build(tdgl_unet *n) {
    const int Lv = n->levels;
    auto add = [&](int ci, int co, int ntap, int lev, bool relu, bool need_dx, int ci_real, int co_real) {
        Layer l;
        l.Ci = ci; l.Co = co; l.ntap = ntap; l.lev = lev; l.relu = relu; l.need_dx = need_dx;
        l.ci_real = ci_real; l.co_real = co_real;
        l.Kp = pad16(ntap * ci);
        l.Kpt = pad16(ntap * co);
        l.ow = n->nparam;
        n->nparam += (size_t)co * l.Kp;
        l.ob = n->nparam;
        n->nparam += (size_t)co;
        n->nflat += (long)co_real * ci_real * ntap + co_real;
        n->L.push_back(l);
    };
    int cprev = 8;    // input channels padded to 8
    for (int l = 0; l < Lv; ++l) {
        const int c = n->chans[l];
        add(cprev, c, 27, l, true, l > 0, l == 0 ? n->cin : cprev, c);
        add(c, c, 27, l, true, true, c, c);
        cprev = c;
    }
    for (int l = Lv - 2; l >= 0; --l) {
        const int c = n->chans[l];
        add(cprev + c, c, 27, l, true, true, cprev + c, c);
        add(c, c, 27, l, true, true, c, c);
        cprev = c;
    }
    add(n->chans[0], n->coutp, 1, 0, false, true, n->chans[0], n->cout);   // output channels padded to 8
    TRY(dalloc(n, &n->P, n->nparam));
    TRY(dalloc(n, &n->G, n->nparam));
    TRY(dalloc(n, &n->M, n->nparam));
    TRY(dalloc(n, &n->V, n->nparam));
    size_t max_dpre = 0, max_xs = 0, max_wpart = 0, max_bpart = 0;
    for (auto &l : n->L) {
        TRY(dalloc(n, &l.wf, (size_t)l.Co * l.Kp));
        TRY(dalloc(n, &l.wt, (size_t)l.Ci * l.Kpt));
        if (l.ntap == 27) {
            TRY(dalloc(n, &l.wfb, (size_t)27 * l.Co * l.Ci));
            TRY(dalloc(n, &l.wtb, (size_t)27 * l.Ci * l.Co));
        }
        const size_t V = (size_t)nvox(n, l.lev, n->maxb);
        max_dpre = std::max(max_dpre, V * l.Co);
        max_xs = std::max(max_xs, 3 * V * l.Ci);
        max_wpart = std::max(max_wpart, wgrad_part_floats((long)V, l.Ci, l.Co, l.ntap, l.Kp));
        max_bpart = std::max(max_bpart, bias_part_floats((long)V, l.Co));
    }
    TRY(dalloc(n, &n->wpart, max_wpart));
    TRY(dalloc(n, &n->bpart, max_bpart));
    // activations: every layer's output, the pooled / concatenated inputs, the input
    const int B = n->maxb;
    TRY(dalloc(n, &n->xin, (size_t)nvox(n, 0, B) * 8));
    std::vector<__nv_bfloat16 *> skip(Lv);
    int li = 0;
    __nv_bfloat16 *cur = n->xin;
    for (int l = 0; l < Lv; ++l) {
        if (l > 0) {
            __nv_bfloat16 *p;
            TRY(dalloc(n, &p, (size_t)nvox(n, l, B) * n->chans[l - 1]));
            cur = p;     // filled by pooling the previous level's output
        }
        for (int s = 0; s < 2; ++s, ++li) {
            Layer &ly = n->L[li];
            ly.in = cur;
            __nv_bfloat16 *o;
            TRY(dalloc(n, &o, (size_t)nvox(n, l, B) * ly.Co));
            ly.out = o;
            cur = o;
        }
        skip[l] = cur;
    }
    for (int l = Lv - 2; l >= 0; --l) {
        __nv_bfloat16 *u;
        TRY(dalloc(n, &u, (size_t)nvox(n, l, B) * n->L[li].Ci));
        cur = u;
        for (int s = 0; s < 2; ++s, ++li) {
            Layer &ly = n->L[li];
            ly.in = cur;
            __nv_bfloat16 *o;
            TRY(dalloc(n, &o, (size_t)nvox(n, l, B) * ly.Co));
            ly.out = o;
            cur = o;
        }
    }
    Layer &hd = n->L[li];
    hd.in = cur;
    TRY(dalloc(n, &n->yout, (size_t)nvox(n, 0, B) * n->coutp));
    hd.out = n->yout;
    // gradients: one FP32 buffer per layer output and per layer input that needs one
    for (auto &l : n->L) {
        TRY(dalloc(n, &l.g_out, (size_t)nvox(n, l.lev, B) * l.Co));
        if (l.need_dx) TRY(dalloc(n, &l.g_in, (size_t)nvox(n, l.lev, B) * l.Ci));
    }
    TRY(dalloc(n, &n->tgt, (size_t)nvox(n, 0, B) * n->coutp));
    TRY(dalloc(n, &n->dpre, max_dpre));
    TRY(dalloc(n, &n->dpret, max_dpre));
    TRY(dalloc(n, &n->xs, max_xs));
    TRY(dalloc(n, &n->dloss, 1));
    TRY(dalloc(n, &n->lpart, (size_t)grid_n(1L << 40)));
    TRY(dalloc(n, &n->derr, 1));
    TRY(dalloc(n, &n->hx, (size_t)nvox(n, 0, B) * std::max(n->cin, n->cout)));
    TRY(dalloc(n, &n->hy, (size_t)nvox(n, 0, B) * std::max(n->cin, n->cout)));
    return TDGL_OK;
}

int refresh_bf16(tdgl_unet *n) {
    for (auto &l : n->L)
        TRY(launch(n->ctx, TDGL_K_UNET, [&] {
            k_wcopy<<<grid_n((long)l.Co * l.Kp), 256, 0, n->ctx->stream>>>(n->P + l.ow, l.wf, l.wt, l.wfb, l.wtb, l.Co,
                                                                            l.Ci, l.ntap, l.Kp, l.Kpt);
        }));
    return TDGL_OK;
}

// x: device float32 [B][cin][Z][Y][X]; leaves the output in n->yout ([V0][cout] FP32)
int forward(tdgl_unet *n, const float *x, int B) {
    tdgl_ctx *ctx = n->ctx;
    const int Lv = n->levels;
    const long V0 = nvox(n, 0, B);
    TRY(launch(ctx, TDGL_K_UNET, [&] {
        k_to_ndhwc<<<grid_n(V0 * 8), 256, 0, ctx->stream>>>(x, n->xin, V0, n->cin, 8, n->dims[0].vps());
    }));
    int li = 0;
    for (int l = 0; l < Lv; ++l) {
        const long V = nvox(n, l, B);
        if (l > 0) {
            const Layer &prev = n->L[li - 1];
            const Dims &d = n->dims[l];
            TRY(launch(ctx, TDGL_K_UNET, [&] {
                k_pool<<<grid_n(V * prev.Co), 256, 0, ctx->stream>>>(reinterpret_cast<const __nv_bfloat16 *>(prev.out),
                                                                     n->L[li].in, V, prev.Co, d.Z, d.Y, d.X);
            }));
        }
        for (int s = 0; s < 2; ++s, ++li) {
            Layer &ly = n->L[li];
            TRY(launch_conv(ctx, ly.in, ly.wf, ly.wfb, n->P + ly.ob, ly.out, V, n->dims[l], ly.Ci, ly.Co, ly.ntap, ly.Kp, true,
                            false, n->derr));
        }
    }
    for (int l = Lv - 2; l >= 0; --l) {
        const long V = nvox(n, l, B);
        const Layer &deep = n->L[li - 1];
        const Layer &skip = n->L[2 * l + 1];
        const Dims &d = n->dims[l];
        TRY(launch(ctx, TDGL_K_UNET, [&] {
            const auto *dpo = reinterpret_cast<const __nv_bfloat16 *>(deep.out);
            const auto *spo = reinterpret_cast<const __nv_bfloat16 *>(skip.out);
            if (deep.Co % 8 == 0 && skip.Co % 8 == 0 && aligned16(dpo) && aligned16(spo) && aligned16(n->L[li].in))
                k_upcat_v<<<grid_n(V * (deep.Co + skip.Co) / 8), 256, 0, ctx->stream>>>(dpo, spo, n->L[li].in, V, deep.Co,
                                                                                        skip.Co, d.Z, d.Y, d.X);
            else
                k_upcat<<<grid_n(V * (deep.Co + skip.Co)), 256, 0, ctx->stream>>>(dpo, spo, n->L[li].in, V, deep.Co, skip.Co,
                                                                                   d.Z, d.Y, d.X);
        }));
        for (int s = 0; s < 2; ++s, ++li) {
            Layer &ly = n->L[li];
            TRY(launch_conv(ctx, ly.in, ly.wf, ly.wfb, n->P + ly.ob, ly.out, V, d, ly.Ci, ly.Co, ly.ntap, ly.Kp, true, false,
                            n->derr));
        }
    }
    Layer &hd = n->L[li];
    return launch_conv(ctx, hd.in, hd.wf, nullptr, n->P + hd.ob, hd.out, V0, n->dims[0], hd.Ci, hd.Co, 1, hd.Kp, false, true,
                       n->derr);
}

// backward of one convolution: g_out (FP32) -> parameter gradients and, if needed, g_in
int conv_backward(tdgl_unet *n, Layer &ly, int B) {
    tdgl_ctx *ctx = n->ctx;
    const long V = nvox(n, ly.lev, B);
    const Dims &d = n->dims[ly.lev];
    float *gw = n->G + ly.ow, *gb = n->G + ly.ob;
    const __nv_bfloat16 *out = ly.relu ? reinterpret_cast<const __nv_bfloat16 *>(ly.out) : nullptr;
    TRY(launch_relu_bwd(ctx, ly.g_out, out, n->dpre, n->dpret, gb, n->bpart, V, ly.Co));
    TRY(launch(ctx, TDGL_K_UNET, [&] {
        k_xshift<<<(unsigned)((V + xshift_vb(ly.Ci) - 1) / xshift_vb(ly.Ci)), 256, xshift_smem(ly.Ci), ctx->stream>>>(
            ly.in, n->xs, V, ly.Ci, d.X, ly.ntap == 27 ? 3 : 1, xshift_vb(ly.Ci));
    }));
    TRY(launch_wgrad(ctx, n->dpret, n->xs, gw, n->wpart, V, d, ly.Ci, ly.Co, ly.ntap, ly.Kp, n->derr));
    if (ly.need_dx)
        TRY(launch_conv(ctx, n->dpre, ly.wt, ly.wtb, nullptr, ly.g_in, V, d, ly.Co, ly.Ci, ly.ntap, ly.Kpt, false, true,
                        n->derr));
    return TDGL_OK;
}

// gradients of the loss (its gradient already in the head's g_out) with respect to every parameter
int backward(tdgl_unet *n, int B) {
    tdgl_ctx *ctx = n->ctx;
    const int Lv = n->levels;
    const int nl = (int)n->L.size();
    auto copy = [&](float *dst, const float *src, size_t count) {
        return cudaMemcpyAsync(dst, src, count * sizeof(float), cudaMemcpyDeviceToDevice, ctx->stream);
    };
    CK(ctx, cudaMemsetAsync(n->G, 0, n->nparam * sizeof(float), ctx->stream));
    Layer &hd = n->L[nl - 1];
    TRY(conv_backward(n, hd, B));
    CK(ctx, copy(n->L[nl - 2].g_out, hd.g_in, (size_t)nvox(n, 0, B) * hd.Ci));
    // decoder, last level first: layers b then a of level l, then split the concatenated input
    // gradient into the deeper part (summed over the 8 children) and the skip part
    int li = nl - 2;
    for (int l = 0; l <= Lv - 2; ++l) {
        Layer &b = n->L[li], &a = n->L[li - 1];
        TRY(conv_backward(n, b, B));
        CK(ctx, copy(a.g_out, b.g_in, (size_t)nvox(n, l, B) * a.Co));
        TRY(conv_backward(n, a, B));
        Layer &deep = n->L[li - 2];            // the layer whose output was upsampled
        Layer &skip = n->L[2 * l + 1];         // encoder level l, layer b
        const Dims &dh = n->dims[l + 1];
        const long Vh = nvox(n, l + 1, B);
        TRY(launch(ctx, TDGL_K_UNET, [&] {
            k_upcat_bwd<<<grid_n(Vh * deep.Co + 8 * Vh * skip.Co), 256, 0, ctx->stream>>>(
                a.g_in, deep.g_out, skip.g_out, Vh, deep.Co, skip.Co, dh.Z, dh.Y, dh.X);
        }));
        li -= 2;
    }
    // encoder, deepest first; g_out of encoder layer b of every level already holds the gradient
    // through the decoder (skip or, at the bottom, the upsampling)
    for (int l = Lv - 1; l >= 0; --l) {
        Layer &b = n->L[2 * l + 1], &a = n->L[2 * l];
        if (l < Lv - 1) {   // + the gradient through the pooling into level l + 1
            const Layer &below = n->L[2 * (l + 1)];
            const Dims &d = n->dims[l];
            const long V = nvox(n, l, B);
            TRY(launch(ctx, TDGL_K_UNET, [&] {
                k_pool_bwd<<<grid_n(V * b.Co), 256, 0, ctx->stream>>>(below.g_in, b.g_out, V, b.Co, d.Z, d.Y, d.X, 1);
            }));
        }
        TRY(conv_backward(n, b, B));
        CK(ctx, copy(a.g_out, b.g_in, (size_t)nvox(n, l, B) * a.Co));
        TRY(conv_backward(n, a, B));
    }
    return TDGL_OK;
}

int stage_in(tdgl_unet *n, const float *src, float *dst, size_t count, int where) {
    if (where == TDGL_DEVICE) return TDGL_OK;
    CK(n->ctx, cudaMemcpyAsync(dst, src, count * sizeof(float), cudaMemcpyHostToDevice, n->ctx->stream));
    return TDGL_OK;
}

// loss and head gradient for target t (device, [B][cout][...])
int loss(tdgl_unet *n, const float *t, int B) {
    tdgl_ctx *ctx = n->ctx;
    const long V0 = nvox(n, 0, B);
    Layer &hd = n->L.back();
    TRY(launch(ctx, TDGL_K_UNET, [&] {
        k_to_ndhwc_f32<<<grid_n(V0 * n->coutp), 256, 0, ctx->stream>>>(t, n->tgt, V0, n->cout, n->coutp,
                                                                          n->dims[0].vps());
    }));
    const int nb = grid_n(V0 * n->coutp);
    TRY(launch(ctx, TDGL_K_UNET, [&] {
        k_mse<<<nb, 256, 0, ctx->stream>>>(n->yout, n->tgt, hd.g_out, V0 * n->coutp, (double)V0 * n->cout, n->lpart);
    }));
    return launch(ctx, TDGL_K_UNET, [&] { k_dsum<<<1, 256, 0, ctx->stream>>>(n->dloss, n->lpart, nb); });
}

int check_batch(tdgl_unet *n, int B) {
    if (B < 1 || B > n->maxb) return fail(n->ctx, TDGL_EINVAL, "batch %d outside 1..%d", B, n->maxb);
    return TDGL_OK;
}

// boundary order <-> GEMM layout: w[o][i][t] <-> W[o][t * Ci + i] (input channels of layer 0
// padded from cin to 8 with zero weights)
void flat_to_gemm(const tdgl_unet *n, const float *flat, std::vector<float> &g) {
    g.assign(n->nparam, 0.f);
    size_t f = 0;
    for (const Layer &l : n->L) {
        for (int o = 0; o < l.co_real; ++o)
            for (int i = 0; i < l.ci_real; ++i)
                for (int t = 0; t < l.ntap; ++t) g[l.ow + (size_t)o * l.Kp + (size_t)t * l.Ci + i] = flat[f++];
        for (int o = 0; o < l.co_real; ++o) g[l.ob + o] = flat[f++];
    }
}
void gemm_to_flat(const tdgl_unet *n, const std::vector<float> &g, float *flat) {
    size_t f = 0;
    for (const Layer &l : n->L) {
        for (int o = 0; o < l.co_real; ++o)
            for (int i = 0; i < l.ci_real; ++i)
                for (int t = 0; t < l.ntap; ++t) flat[f++] = g[l.ow + (size_t)o * l.Kp + (size_t)t * l.Ci + i];
        for (int o = 0; o < l.co_real; ++o) flat[f++] = g[l.ob + o];
    }
}

}  // namespace

extern "C" {

int tdgl_unet_create(tdgl_ctx *ctx, int cin, int cout, int levels, const int *chans, int nx, int ny, int nz,
                     int max_batch, uint64_t seed, tdgl_unet **out) {
    if (!ctx || !out || !chans) return fail(ctx, TDGL_EINVAL, "null argument");
    *out = nullptr;
    if (cin < 1 || cin > 8 || cout < 1 || cout > 16 || levels < 2 || levels > 5 || max_batch < 1)
        return fail(ctx, TDGL_EINVAL, "unet: cin 1..8, cout 1..16, levels 2..5, max_batch >= 1");
    const int f = 1 << (levels - 1);
    if (nx % (8 * f) || ny % f || nz % f || nx <= 0 || ny <= 0 || nz <= 0)
        return fail(ctx, TDGL_EINVAL, "unet: nx must be a multiple of %d and ny, nz of %d", 8 * f, f);
    for (int l = 0; l < levels; ++l)
        if (chans[l] < 16 || chans[l] > 128 || chans[l] % 16)
            return fail(ctx, TDGL_EINVAL, "unet: channels must be multiples of 16 in 16..128");
    ctx_set(ctx);
    TRY(init_attrs(ctx));
    tdgl_unet *n = new tdgl_unet();
    n->ctx = ctx;
    n->cin = cin; n->cout = cout; n->coutp = (cout + 7) & ~7; n->levels = levels; n->maxb = max_batch;
    for (int l = 0; l < levels; ++l) {
        n->chans[l] = chans[l];
        n->dims[l] = Dims{nz >> l, ny >> l, nx >> l};
    }
    int rc = build(n);
    if (rc == TDGL_OK) {
        // He-normal weights: std sqrt(2 / fan_in), fan_in = real input channels x taps; the padded
        // input channels of layer 0 and output rows of the head are drawn, then zeroed
        for (size_t k = 0; k < n->L.size() && rc == TDGL_OK; ++k) {
            Layer &l = n->L[k];
            const float sd = (float)sqrt(2.0 / ((double)l.ci_real * l.ntap));
            rc = launch(ctx, TDGL_K_UNET, [&] {
                k_init_he<<<grid_n((long)l.Co * l.Kp), 256, 0, ctx->stream>>>(
                    n->P + l.ow, l.Co, l.Kp, l.ntap * l.Ci, sd, (uint32_t)k, (uint32_t)seed, (uint32_t)(seed >> 32));
            });
            if (rc == TDGL_OK && (l.ci_real != l.Ci || l.co_real != l.Co)) {
                std::vector<float> w((size_t)l.Co * l.Kp);
                cudaMemcpyAsync(w.data(), n->P + l.ow, w.size() * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream);
                cudaStreamSynchronize(ctx->stream);
                for (int o = 0; o < l.Co; ++o)
                    for (int t = 0; t < l.ntap; ++t)
                        for (int i = 0; i < l.Ci; ++i)
                            if (o >= l.co_real || i >= l.ci_real) w[(size_t)o * l.Kp + (size_t)t * l.Ci + i] = 0.f;
                cudaMemcpyAsync(n->P + l.ow, w.data(), w.size() * sizeof(float), cudaMemcpyHostToDevice, ctx->stream);
                cudaStreamSynchronize(ctx->stream);
            }
        }
        if (rc == TDGL_OK) rc = refresh_bf16(n);
        if (rc == TDGL_OK) {
            cudaError_t e = cudaStreamSynchronize(ctx->stream);
            if (e != cudaSuccess) rc = fail(ctx, TDGL_ECUDA, "unet init: %s", cudaGetErrorString(e));
        }
    }
    if (rc != TDGL_OK) {
        for (void *p : n->bufs) cudaFree(p);
        delete n;
        return rc;
    }
    ctx->nets.push_back(n);
    *out = n;
    return TDGL_OK;
}

void tdgl_unet_destroy(tdgl_unet *n) {
    if (!n) return;
    ctx_set(n->ctx);
    cudaStreamSynchronize(n->ctx->stream);
    auto &v = n->ctx->nets;
    v.erase(std::remove(v.begin(), v.end(), n), v.end());
    for (void *p : n->bufs) cudaFree(p);
    delete n;
}

long tdgl_unet_param_count(const tdgl_unet *n) { return n ? n->nflat : 0; }

int tdgl_unet_set_params(tdgl_unet *n, const float *params) {
    if (!n || !params) return TDGL_EINVAL;
    ctx_set(n->ctx);
    std::vector<float> g;
    flat_to_gemm(n, params, g);
    CK(n->ctx, cudaMemcpyAsync(n->P, g.data(), g.size() * sizeof(float), cudaMemcpyHostToDevice, n->ctx->stream));
    CK(n->ctx, cudaMemsetAsync(n->M, 0, n->nparam * sizeof(float), n->ctx->stream));
    CK(n->ctx, cudaMemsetAsync(n->V, 0, n->nparam * sizeof(float), n->ctx->stream));
    n->step = 0;
    TRY(refresh_bf16(n));
    CK(n->ctx, cudaStreamSynchronize(n->ctx->stream));
    return TDGL_OK;
}

int tdgl_unet_get_params(tdgl_unet *n, float *params) {
    if (!n || !params) return TDGL_EINVAL;
    ctx_set(n->ctx);
    std::vector<float> g(n->nparam);
    CK(n->ctx, cudaMemcpyAsync(g.data(), n->P, g.size() * sizeof(float), cudaMemcpyDeviceToHost, n->ctx->stream));
    CK(n->ctx, cudaStreamSynchronize(n->ctx->stream));
    gemm_to_flat(n, g, params);
    return TDGL_OK;
}

int tdgl_unet_forward(tdgl_unet *n, const float *x, float *y, int batch, int where) {
    if (!n || !x || !y) return TDGL_EINVAL;
    TRY(check_batch(n, batch));
    ctx_set(n->ctx);
    tdgl_ctx *ctx = n->ctx;
    const long V0 = nvox(n, 0, batch);
    const float *dx = x;
    if (where == TDGL_HOST) {
        TRY(stage_in(n, x, n->hx, (size_t)V0 * n->cin, where));
        dx = n->hx;
    }
    TRY(forward(n, dx, batch));
    float *dy = (where == TDGL_HOST) ? n->hy : y;
    TRY(launch(ctx, TDGL_K_UNET, [&] {
        k_from_ndhwc_f32<<<grid_n(V0 * n->cout), 256, 0, ctx->stream>>>(n->yout, dy, V0, n->cout, n->coutp,
                                                                          n->dims[0].vps());
    }));
    if (where == TDGL_HOST)
        CK(ctx, cudaMemcpyAsync(y, n->hy, (size_t)V0 * n->cout * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    return check_err(ctx, n->derr);
}

}  // extern "C"

static int loss_and_grads(tdgl_unet *n, const float *x, const float *t, int batch, double *loss_out, int where) {
    tdgl_ctx *ctx = n->ctx;
    const long V0 = nvox(n, 0, batch);
    const float *dx = x, *dt = t;
    if (where == TDGL_HOST) {
        TRY(stage_in(n, x, n->hx, (size_t)V0 * n->cin, where));
        TRY(stage_in(n, t, n->hy, (size_t)V0 * n->cout, where));
        dx = n->hx;
        dt = n->hy;
    }
    TRY(forward(n, dx, batch));
    TRY(loss(n, dt, batch));
    TRY(backward(n, batch));
    if (loss_out) CK(ctx, cudaMemcpyAsync(loss_out, n->dloss, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    return TDGL_OK;
}

extern "C" {

int tdgl_unet_loss_grad(tdgl_unet *n, const float *x, const float *t, int batch, double *loss_out, float *grads,
                        int where) {
    if (!n || !x || !t || !grads) return TDGL_EINVAL;
    TRY(check_batch(n, batch));
    ctx_set(n->ctx);
    TRY(loss_and_grads(n, x, t, batch, loss_out, where));
    std::vector<float> g(n->nparam);
    CK(n->ctx, cudaMemcpyAsync(g.data(), n->G, g.size() * sizeof(float), cudaMemcpyDeviceToHost, n->ctx->stream));
    TRY(check_err(n->ctx, n->derr));
    gemm_to_flat(n, g, grads);
    return TDGL_OK;
}

int tdgl_unet_train_step(tdgl_unet *n, const float *x, const float *t, int batch, double lr, double *loss_out,
                         int where) {
    if (!n || !x || !t || !(lr > 0)) return TDGL_EINVAL;
    TRY(check_batch(n, batch));
    ctx_set(n->ctx);
    tdgl_ctx *ctx = n->ctx;
    TRY(loss_and_grads(n, x, t, batch, loss_out, where));
    n->step++;
    const double b1 = 0.9, b2 = 0.999;
    for (auto &l : n->L) {
        AdamP p{n->P + l.ow, n->M + l.ow, n->V + l.ow, n->G + l.ow, n->P + l.ob, n->M + l.ob, n->V + l.ob, n->G + l.ob,
                l.wf, l.wt, l.wfb, l.wtb, l.Co, l.Ci, l.ntap, l.Kp, l.Kpt, (float)lr, (float)b1, (float)b2, 1e-8f,
                (float)(1.0 - pow(b1, (double)n->step)), (float)(1.0 - pow(b2, (double)n->step))};
        TRY(launch(ctx, TDGL_K_UNET, [&] { k_adam<<<grid_n((long)l.Co * l.Kp + l.Co), 256, 0, ctx->stream>>>(p); }));
    }
    return check_err(ctx, n->derr);
}

}  // extern "C"

// ---- single convolutions ------------------------------------------------------------------------

namespace {
struct Scratch {
    std::vector<void *> p;
    ~Scratch() {
        for (void *q : p) cudaFree(q);
    }
    template <class T>
    int get(tdgl_ctx *ctx, T **out, size_t n) {
        void *q = nullptr;
        CK(ctx, cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T)));
        CK(ctx, cudaMemsetAsync(q, 0, std::max<size_t>(n, 1) * sizeof(T), ctx->stream));
        p.push_back(q);
        *out = reinterpret_cast<T *>(q);
        return TDGL_OK;
    }
};

int conv_check(tdgl_ctx *ctx, int batch, int ci, int co, int k, int nx, int ny, int nz) {
    if (batch < 1 || ci < 8 || ci % 8 || ci > 192 || co < 1 || co > 128 || (k != 1 && k != 3) || nx % 8 || nx <= 0 ||
        ny <= 0 || nz <= 0)
        return fail(ctx, TDGL_EINVAL, "conv3d: ci multiple of 8 (<= 192), co 1..128, k 1 or 3, nx multiple of 8");
    return TDGL_OK;
}

// weights [co][ci][t] (host) -> device GEMM layouts: FP32 master [co][Kp], BF16 forward and transposed
int upload_w(tdgl_ctx *ctx, Scratch &S, const float *w, int ci, int co, int ntap, float **wm, __nv_bfloat16 **wf,
             __nv_bfloat16 **wt, __nv_bfloat16 **wfb, __nv_bfloat16 **wtb, int *Kp, int *Kpt) {
    *Kp = pad16(ntap * ci);
    *Kpt = pad16(ntap * co);
    std::vector<float> g((size_t)co * *Kp, 0.f);
    for (int o = 0; o < co; ++o)
        for (int i = 0; i < ci; ++i)
            for (int t = 0; t < ntap; ++t) g[(size_t)o * *Kp + (size_t)t * ci + i] = w[((size_t)o * ci + i) * ntap + t];
    TRY(S.get(ctx, wm, g.size()));
    TRY(S.get(ctx, wf, g.size()));
    TRY(S.get(ctx, wt, (size_t)ci * *Kpt));
    *wfb = *wtb = nullptr;
    if (ntap == 27) {
        TRY(S.get(ctx, wfb, (size_t)27 * co * ci));
        TRY(S.get(ctx, wtb, (size_t)27 * ci * co));
    }
    CK(ctx, cudaMemcpyAsync(*wm, g.data(), g.size() * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    return launch(ctx, TDGL_K_UNET, [&] {
        k_wcopy<<<grid_n((long)co * *Kp), 256, 0, ctx->stream>>>(*wm, *wf, *wt, *wfb, *wtb, co, ci, ntap, *Kp, *Kpt);
    });
}
}  // namespace

extern "C" {

int tdgl_conv3d(tdgl_ctx *ctx, const float *x, const float *w, const float *b, float *y, int batch, int ci, int co,
                int k, int nx, int ny, int nz, int relu) {
    if (!ctx || !x || !w || !y) return fail(ctx, TDGL_EINVAL, "null argument");
    TRY(conv_check(ctx, batch, ci, co, k, nx, ny, nz));
    ctx_set(ctx);
    TRY(init_attrs(ctx));
    Scratch S;
    const int ntap = k * k * k;
    const Dims d{nz, ny, nx};
    const long V = (long)batch * d.vps();
    float *dx, *db = nullptr, *dy, *dy2, *wm;
    __nv_bfloat16 *xb, *wf, *wt, *wfb, *wtb;
    int Kp, Kpt, *derr;
    TRY(S.get(ctx, &dx, (size_t)V * ci));
    TRY(S.get(ctx, &xb, (size_t)V * ci));
    TRY(S.get(ctx, &dy, (size_t)V * co));
    TRY(S.get(ctx, &dy2, (size_t)V * co));
    TRY(S.get(ctx, &derr, 1));
    CK(ctx, cudaMemcpyAsync(dx, x, (size_t)V * ci * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    TRY(launch(ctx, TDGL_K_UNET, [&] { k_to_ndhwc<<<grid_n(V * ci), 256, 0, ctx->stream>>>(dx, xb, V, ci, ci, d.vps()); }));
    TRY(upload_w(ctx, S, w, ci, co, ntap, &wm, &wf, &wt, &wfb, &wtb, &Kp, &Kpt));
    if (b) {
        TRY(S.get(ctx, &db, (size_t)co));
        CK(ctx, cudaMemcpyAsync(db, b, co * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    }
    TRY(launch_conv(ctx, xb, wf, wfb, db, dy, V, d, ci, co, ntap, Kp, relu != 0, true, derr));
    TRY(launch(ctx, TDGL_K_UNET, [&] { k_from_ndhwc_f32<<<grid_n(V * co), 256, 0, ctx->stream>>>(dy, dy2, V, co, co, d.vps()); }));
    CK(ctx, cudaMemcpyAsync(y, dy2, (size_t)V * co * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    return check_err(ctx, derr);
}

int tdgl_conv3d_backward(tdgl_ctx *ctx, const float *x, const float *w, const float *dyh, float *dxh, float *dwh,
                         float *dbh, int batch, int ci, int co, int k, int nx, int ny, int nz) {
    if (!ctx || !x || !w || !dyh || !dxh || !dwh || !dbh) return fail(ctx, TDGL_EINVAL, "null argument");
    TRY(conv_check(ctx, batch, ci, co, k, nx, ny, nz));
    if (co % 8) return fail(ctx, TDGL_EINVAL, "conv3d_backward: co must be a multiple of 8");
    ctx_set(ctx);
    TRY(init_attrs(ctx));
    Scratch S;
    const int ntap = k * k * k;
    const Dims d{nz, ny, nx};
    const long V = (long)batch * d.vps();
    float *xf, *gy, *gyn, *gx, *gxo, *wm, *gw, *gb, *wpart, *bpart;
    __nv_bfloat16 *xb, *wf, *wt, *wfb, *wtb, *dpre, *dpret, *xs;
    int Kp, Kpt, *derr;
    TRY(S.get(ctx, &xf, (size_t)V * ci));
    TRY(S.get(ctx, &xb, (size_t)V * ci));
    TRY(S.get(ctx, &gy, (size_t)V * co));
    TRY(S.get(ctx, &gyn, (size_t)V * co));
    TRY(S.get(ctx, &gx, (size_t)V * ci));
    TRY(S.get(ctx, &gxo, (size_t)V * ci));
    TRY(S.get(ctx, &dpre, (size_t)V * co));
    TRY(S.get(ctx, &dpret, (size_t)V * co));
    TRY(S.get(ctx, &xs, (size_t)3 * V * ci));
    TRY(S.get(ctx, &derr, 1));
    TRY(upload_w(ctx, S, w, ci, co, ntap, &wm, &wf, &wt, &wfb, &wtb, &Kp, &Kpt));
    TRY(S.get(ctx, &gw, (size_t)co * Kp));
    TRY(S.get(ctx, &gb, (size_t)co));
    TRY(S.get(ctx, &wpart, wgrad_part_floats(V, ci, co, ntap, Kp)));
    TRY(S.get(ctx, &bpart, bias_part_floats(V, co)));
    CK(ctx, cudaMemcpyAsync(xf, x, (size_t)V * ci * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    CK(ctx, cudaMemcpyAsync(gy, dyh, (size_t)V * co * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    TRY(launch(ctx, TDGL_K_UNET, [&] { k_to_ndhwc<<<grid_n(V * ci), 256, 0, ctx->stream>>>(xf, xb, V, ci, ci, d.vps()); }));
    TRY(launch(ctx, TDGL_K_UNET, [&] { k_to_ndhwc_f32<<<grid_n(V * co), 256, 0, ctx->stream>>>(gy, gyn, V, co, co, d.vps()); }));
    TRY(launch_relu_bwd(ctx, gyn, nullptr, dpre, dpret, gb, bpart, V, co));
    TRY(launch(ctx, TDGL_K_UNET, [&] {
        k_xshift<<<(unsigned)((V + xshift_vb(ci) - 1) / xshift_vb(ci)), 256, xshift_smem(ci), ctx->stream>>>(
            xb, xs, V, ci, d.X, ntap == 27 ? 3 : 1, xshift_vb(ci));
    }));
    TRY(launch_wgrad(ctx, dpret, xs, gw, wpart, V, d, ci, co, ntap, Kp, derr));
    TRY(launch_conv(ctx, dpre, wt, wtb, nullptr, gx, V, d, co, ci, ntap, Kpt, false, true, derr));
    TRY(launch(ctx, TDGL_K_UNET, [&] { k_from_ndhwc_f32<<<grid_n(V * ci), 256, 0, ctx->stream>>>(gx, gxo, V, ci, ci, d.vps()); }));
    std::vector<float> g((size_t)co * Kp);
    CK(ctx, cudaMemcpyAsync(dxh, gxo, (size_t)V * ci * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaMemcpyAsync(g.data(), gw, g.size() * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaMemcpyAsync(dbh, gb, co * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    TRY(check_err(ctx, derr));
    for (int o = 0; o < co; ++o)
        for (int i = 0; i < ci; ++i)
            for (int t = 0; t < ntap; ++t) dwh[((size_t)o * ci + i) * ntap + t] = g[(size_t)o * Kp + (size_t)t * ci + i];
    return TDGL_OK;
}

}  // extern "C"
