// Internal runtime shared by the library's translation units: the context object, error
// reporting and the counted (optionally event-timed) kernel launch.  Not part of the C ABI.
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/tdgl.h"

struct tdgl_sim;
struct tdgl_batch;
struct tdgl_unet;

namespace tdgl_rt {

struct ProfRec {
    int kind;
    cudaEvent_t a, b;
};

}  // namespace tdgl_rt

struct tdgl_ctx {
    int device = 0;
    int nsm = 148;                      // streaming multiprocessors of the device
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // copy streams of the asynchronous host I/O calls (created on first use): uploads, downloads
    cudaStream_t up = nullptr, down = nullptr;
    // split-K partial sums of the network's small convolutions (grown on demand, reused by every
    // convolution of the context: its work is ordered on the one stream)
    float *splitk = nullptr;
    size_t splitk_n = 0;
    std::string err;
    long launches = 0;
    bool profiling = false;
    std::vector<tdgl_rt::ProfRec> recs;
    std::vector<cudaEvent_t> pool;
    double prof_ms[TDGL_K_COUNT] = {0};
    long prof_n[TDGL_K_COUNT] = {0};
    std::vector<tdgl_sim *> sims;       // owned: freed by tdgl_ctx_destroy if still alive
    std::vector<tdgl_batch *> batches;
    std::vector<tdgl_unet *> nets;
    // z-pass radix-schedule autotuning for 256-, 512- and 128-point lines (in that index order): chosen variant (-1 = not
    // yet tuned) and the measured microseconds per launch of each variant
    int zvar[3] = {-1, -1, -1};
    double zus[3][TDGL_ZPASS_VARIANTS] = {};
    // row-tile autotuning of sims run alone, per (x half-length, ny, nz, electrostatics on): the
    // chosen rows per block and the candidates' timings
    struct RowTune {
        int hx, ny, nz, elec, tile;
        int cand[TDGL_ROW_CANDIDATES];
        double us[TDGL_ROW_CANDIDATES];
    };
    std::vector<RowTune> rowtune;
};

namespace tdgl_rt {

inline int fail(tdgl_ctx *ctx, int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (ctx) ctx->err = buf;
    return code;
}

#define CK(ctx, call)                                                                            \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess)                                                                   \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? TDGL_ENOMEM : TDGL_ECUDA,         \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__);   \
    } while (0)

#define TRY(x)                  \
    do {                        \
        int r_ = (x);           \
        if (r_ != TDGL_OK) return r_; \
    } while (0)

inline void ctx_set(tdgl_ctx *ctx) { cudaSetDevice(ctx->device); }

inline cudaEvent_t take_event(tdgl_ctx *ctx) {
    if (!ctx->pool.empty()) {
        cudaEvent_t e = ctx->pool.back();
        ctx->pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

// launch through f() on the context's stream: counted, timed when profiling is on, checked
template <class F>
inline int launch(tdgl_ctx *ctx, int kind, F f) {
    ProfRec r{kind, nullptr, nullptr};
    if (ctx->profiling) {
        r.a = take_event(ctx);
        r.b = take_event(ctx);
        cudaEventRecord(r.a, ctx->stream);
    }
    f();
    cudaError_t e = cudaGetLastError();
    if (ctx->profiling) {
        cudaEventRecord(r.b, ctx->stream);
        ctx->recs.push_back(r);
    }
    ctx->launches++;
    if (e != cudaSuccess) return fail(ctx, TDGL_ECUDA, "kernel launch (kind %d): %s", kind, cudaGetErrorString(e));
    return TDGL_OK;
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime (null if unavailable)
inline PFN_cuTensorMapEncodeTiled_v12000 tmap_encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    }
    return fn;
}

}  // namespace tdgl_rt
