// Context life cycle, status reporting, workspace pool and the link import (canonical complex128
// [V][4][3][3] -> FP64 structure-of-arrays + FP32 two-row / third-row arrays).
#include <stdarg.h>
#include <algorithm>
#include <string.h>

#include "common.cuh"

namespace rm {

int set_err(rmhmc_ctx* ctx, int code, const char* fmt, ...) {
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return code;
}

int cuda_check(rmhmc_ctx* ctx, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return RMHMC_OK;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return set_err(ctx, RMHMC_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
    }
    return set_err(ctx, RMHMC_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

void* workspace(rmhmc_ctx* ctx, const char* name, size_t bytes, int* status) {
    DevBuf& b = ctx->bufs[name];
    if (b.bytes >= bytes && b.p) return b.p;
    if (b.p) {
        cudaDeviceSynchronize();
        cudaFree(b.p);
        b.p = nullptr;
        b.bytes = 0;
    }
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        *status = cuda_check(ctx, e, name);
        return nullptr;
    }
    b.p = p;
    b.bytes = bytes;
    ctx->ws_gen++;
    return p;
}

double* red_slot_partials(rmhmc_ctx* ctx, int slot) { return ctx->red_partials + (size_t)slot * ctx->max_blocks * 2; }
unsigned* red_slot_counter(rmhmc_ctx* ctx, int slot) { return ctx->red_counters + slot; }
double* red_slot_out(rmhmc_ctx* ctx, int slot) { return ctx->red_out + (size_t)slot * 8; }

int upload(rmhmc_ctx* ctx, void* dst, const void* src, size_t bytes, cudaStream_t st) {
    if (bytes > kRingBytes) return set_err(ctx, RMHMC_EINVAL, "upload of %zu bytes exceeds the staging slot", bytes);
    const unsigned slot = ctx->ring_idx++ % kRingSlots;
    RM_CHECK(ctx, cudaEventSynchronize(ctx->ring_ev[slot]));
    char* hp = ctx->ring + (size_t)slot * kRingBytes;
    memcpy(hp, src, bytes);
    RM_CHECK(ctx, cudaMemcpyAsync(dst, hp, bytes, cudaMemcpyHostToDevice, st));
    RM_CHECK(ctx, cudaEventRecord(ctx->ring_ev[slot], st));
    return RMHMC_OK;
}

int fetch(rmhmc_ctx* ctx, const double* dsrc, double* hdst, int n, cudaStream_t st) {
    if (n > kPinned) return set_err(ctx, RMHMC_EINVAL, "fetch of %d doubles exceeds the staging area", n);
    RM_CHECK(ctx, cudaMemcpyAsync(ctx->h_pinned, dsrc, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
    RM_CHECK(ctx, cudaStreamSynchronize(st));
    memcpy(hdst, ctx->h_pinned, sizeof(double) * n);
    return RMHMC_OK;
}

__global__ void k_import_links(const double* __restrict__ U, double2* __restrict__ u64, float4* __restrict__ u32a,
                               float2* __restrict__ u32b, int V) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= V) return;
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
        const double2* src = reinterpret_cast<const double2*>(U + ((size_t)s * 4 + mu) * 18);
        double2 e[9];
#pragma unroll
        for (int k = 0; k < 9; k++) e[k] = src[k];
#pragma unroll
        for (int k = 0; k < 9; k++) u64[(size_t)(mu * 9 + k) * V + s] = e[k];
        u32a[(size_t)(mu * 3 + 0) * V + s] = make_float4((float)e[0].x, (float)e[0].y, (float)e[1].x, (float)e[1].y);
        u32a[(size_t)(mu * 3 + 1) * V + s] = make_float4((float)e[2].x, (float)e[2].y, (float)e[3].x, (float)e[3].y);
        u32a[(size_t)(mu * 3 + 2) * V + s] = make_float4((float)e[4].x, (float)e[4].y, (float)e[5].x, (float)e[5].y);
#pragma unroll
        for (int j = 0; j < 3; j++) u32b[(size_t)(mu * 3 + j) * V + s] = make_float2((float)e[6 + j].x, (float)e[6 + j].y);
    }
}

int import_links(rmhmc_ctx* ctx, const double* U, cudaStream_t st) {
    if (((uintptr_t)U) % 16) return set_err(ctx, RMHMC_EINVAL, "links must be 16-byte aligned");
    k_import_links<<<site_blocks(ctx), kBlock, 0, st>>>(U, ctx->u64, ctx->u32a, ctx->u32b, ctx->g.V); ++ctx->launches;
    RM_LAUNCH_CHECK(ctx);
    ctx->links_valid = true;
    ctx->link_gen++;
    return RMHMC_OK;
}

int ensure_links(rmhmc_ctx* ctx, const double* U, cudaStream_t st) {
    if (U) return import_links(ctx, U, st);
    if (!ctx->links_valid) return set_err(ctx, RMHMC_EINVAL, "no links: pass U or call rmhmc_set_links first");
    return RMHMC_OK;
}

}  // namespace rm

using namespace rm;

extern "C" int rmhmc_create(const int dims[4], int device, rmhmc_ctx** out) {
    if (!dims || !out) return RMHMC_EINVAL;
    *out = nullptr;
    // every partial product is checked against the limit, so no extent can overflow the product
    long long V = 1;
    for (int d = 0; d < 4; d++) {
        if (dims[d] < 2 || dims[d] > (1 << 26)) return RMHMC_EINVAL;
        V *= dims[d];
        if (V > (1ll << 26)) return RMHMC_EINVAL;   // site indices stay well inside int
    }
    if (cudaSetDevice(device) != cudaSuccess) return RMHMC_ECUDA;
    rmhmc_ctx* ctx = new rmhmc_ctx();
    ctx->device = device;
    for (int d = 0; d < 4; d++) ctx->g.L[d] = dims[d];
    ctx->g.stride[0] = 1;
    for (int d = 1; d < 4; d++) ctx->g.stride[d] = ctx->g.stride[d - 1] * dims[d - 1];
    ctx->g.V = (int)V;
    geom_init_divmod(ctx->g);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    ctx->num_sms = sms;
    // the most blocks any reduced launch uses: four lanes per site in blocks of kBlockMin, or one float32
    // float4 per thread (8 per site) in blocks of kBlock
    ctx->max_blocks = (int)std::max((4 * V + kBlockMin - 1) / kBlockMin, (8 * V + kBlock - 1) / kBlock);
    cudaError_t e = cudaSuccess;
    e = cudaMalloc(&ctx->u64, sizeof(double2) * 36 * (size_t)V);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->u32a, sizeof(float4) * 12 * (size_t)V);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->u32b, sizeof(float2) * 12 * (size_t)V);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->red_partials, sizeof(double) * kRedSlots * (size_t)ctx->max_blocks * 2);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->red_counters, sizeof(unsigned) * kRedSlots);
    if (e == cudaSuccess) e = cudaMemset(ctx->red_counters, 0, sizeof(unsigned) * kRedSlots);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->red_out, sizeof(double) * kRedSlots * 8);
    if (e == cudaSuccess) e = cudaMallocHost(&ctx->h_pinned, sizeof(double) * kPinned);
    if (e == cudaSuccess) e = cudaMallocHost(&ctx->ring, kRingBytes * kRingSlots);
    for (int i = 0; i < kRingSlots && e == cudaSuccess; i++) e = cudaEventCreateWithFlags(&ctx->ring_ev[i], cudaEventDisableTiming);
    for (int i = 0; i < 2 && e == cudaSuccess; i++) e = cudaEventCreateWithFlags(&ctx->kr_ev[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        rmhmc_destroy(ctx);
        return e == cudaErrorMemoryAllocation ? RMHMC_ENOMEM : RMHMC_ECUDA;
    }
    *out = ctx;
    return RMHMC_OK;
}

extern "C" int rmhmc_destroy(rmhmc_ctx* ctx) {
    if (!ctx) return RMHMC_OK;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    cudaFree(ctx->u64);
    cudaFree(ctx->u32a);
    cudaFree(ctx->u32b);
    cudaFree(ctx->red_partials);
    cudaFree(ctx->red_counters);
    cudaFree(ctx->red_out);
    if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
    if (ctx->ring) cudaFreeHost(ctx->ring);
    for (int i = 0; i < kRingSlots; i++) if (ctx->ring_ev[i]) cudaEventDestroy(ctx->ring_ev[i]);
    for (int i = 0; i < 2; i++) if (ctx->kr_ev[i]) cudaEventDestroy(ctx->kr_ev[i]);
    for (auto& kv : ctx->bufs) cudaFree(kv.second.p);
    if (ctx->md_exec) cudaGraphExecDestroy(ctx->md_exec);
    for (int i = 0; i < 3; i++)
        if (ctx->cap_st[i]) cudaStreamDestroy(ctx->cap_st[i]);
    if (ctx->prof_ev) {
        for (int i = 0; i < 2 * kProfEvents; i++) cudaEventDestroy(ctx->prof_ev[i]);
        delete[] ctx->prof_ev;
    }
    delete ctx;
    return RMHMC_OK;
}

extern "C" const char* rmhmc_last_error(const rmhmc_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

extern "C" int rmhmc_set_links(rmhmc_ctx* ctx, const double* U, cudaStream_t stream) {
    if (!ctx || !U) return set_err(ctx, RMHMC_EINVAL, "rmhmc_set_links: null argument");
    ctx->err.clear();
    return import_links(ctx, U, stream);
}

extern "C" int rmhmc_set_profiling(rmhmc_ctx* ctx, int on) {
    if (!ctx) return RMHMC_EINVAL;
    if (on && !ctx->prof_ev) {
        ctx->prof_ev = new cudaEvent_t[2 * kProfEvents];
        for (int i = 0; i < 2 * kProfEvents; i++)
            if (cudaEventCreate(&ctx->prof_ev[i]) != cudaSuccess) return set_err(ctx, RMHMC_ECUDA, "event creation failed");
    }
    ctx->prof = on != 0;
    return RMHMC_OK;
}

extern "C" int rmhmc_get_counters(rmhmc_ctx* ctx, long long* launches, long long* krylov_iters, long long* cg_count,
                                  double* cg_ms, int reset) {
    if (!ctx) return RMHMC_EINVAL;
    if (launches) *launches = ctx->launches;
    if (krylov_iters) *krylov_iters = ctx->krylov_iters;
    if (cg_count) *cg_count = ctx->prof_count;
    if (cg_ms) *cg_ms = ctx->prof_ms;
    if (reset) {
        ctx->launches = 0;
        ctx->krylov_iters = 0;
        ctx->prof_count = 0;
        ctx->prof_ms = 0.0;
    }
    return RMHMC_OK;
}

extern "C" int rmhmc_tuning(const rmhmc_ctx* ctx, char* buf, int len) {
    if (!ctx || !buf || len < 1) return RMHMC_EINVAL;
    snprintf(buf, (size_t)len, "%s; graphs: %s%s", ctx->tune_report.c_str(), ctx->use_graphs ? "on" : "off",
             ctx->graph_note.empty() ? "" : (" (" + ctx->graph_note + ")").c_str());
    return RMHMC_OK;
}

extern "C" int rmhmc_set_stencil_shape(rmhmc_ctx* ctx, int kernel, int prec, int linkfmt, int nmu, int block) {
    if (!ctx) return RMHMC_EINVAL;
    ctx->err.clear();
    ctx->shape_gen++;
    if (kernel == RMHMC_SHAPE_LINKUPDATE) {
        if (prec != RMHMC_FP64 || linkfmt != 18 || (nmu != 0 && nmu != 1) || block != 128)
            return set_err(ctx, RMHMC_EINVAL, "link update: RMHMC_FP64, 18, nmu 0 or 1, block 128");
        ctx->link_update_ff = nmu == 1;
        return RMHMC_OK;
    }
    if (kernel == RMHMC_SHAPE_KFORCE) {
        if (prec != RMHMC_FP32 || linkfmt != 18 || nmu < 0 || nmu > 3 || block != (nmu == 2 ? 256 : 128))
            return set_err(ctx, RMHMC_EINVAL,
                           "kinetic-force contraction: RMHMC_FP32, 18, nmu 0/1/3 with block 128 or 2 with 256");
        ctx->lg_mode = nmu;
        return RMHMC_OK;
    }
    if (kernel == RMHMC_SHAPE_ADJOINT) {
        if (prec != RMHMC_FP32 || (linkfmt != 12 && linkfmt != 18) || (nmu != 0 && nmu != 2 && nmu != 3) ||
            block < 0 || block > ctx->g.L[2])
            return set_err(ctx, RMHMC_EINVAL, "adjoint kernel: RMHMC_FP32, 12 or 18, nmu 0/2/3, block 0..L2");
        const int key = 20000 + linkfmt;
        if (nmu == 0) ctx->tune.erase(key);
        else ctx->tune[key] = {nmu - 2, 0};
        ctx->ad_slab = block;
        char line[96];
        snprintf(line, sizeof line, "%sadjoint LF%d pinned -> %d fields/pass, slab depth %d",
                 ctx->tune_report.empty() ? "" : "; ", linkfmt, nmu, block);
        ctx->tune_report += line;
        return RMHMC_OK;
    }
    if (kernel != RMHMC_SHAPE_LAP && kernel != RMHMC_SHAPE_CG) return set_err(ctx, RMHMC_EINVAL, "bad kernel");
    if (prec != RMHMC_FP64 && prec != RMHMC_FP32) return set_err(ctx, RMHMC_EINVAL, "bad prec");
    if (linkfmt != 18 && (linkfmt != 12 || kernel == RMHMC_SHAPE_CG)) return set_err(ctx, RMHMC_EINVAL, "bad linkfmt");
    if (nmu != 0 && nmu != 1 && nmu != 2 && nmu != 4 && nmu != 8) return set_err(ctx, RMHMC_EINVAL, "bad nmu");
    if (block != 64 && block != 128 && block != 256) return set_err(ctx, RMHMC_EINVAL, "bad block");
    if (nmu == 8 && (prec != RMHMC_FP32 || block != 256))
        return set_err(ctx, RMHMC_EINVAL, "the link-centric kernel is float32 with 256 threads");
    const int bytes = prec == RMHMC_FP64 ? 8 : 4;
    const int key = (kernel == RMHMC_SHAPE_CG ? 10000 : 0) + bytes * 100 + linkfmt;
    if (kernel == RMHMC_SHAPE_CG && !ctx->tune.count(bytes * 100 + 18)) ctx->tune[bytes * 100 + 18] = {2, 256};
    ctx->tune[key] = {nmu, block};
    char line[96];
    snprintf(line, sizeof line, "%s%s %s LF%d pinned -> nmu %d block %d", ctx->tune_report.empty() ? "" : "; ",
             kernel == RMHMC_SHAPE_CG ? "cg" : "lap", bytes == 8 ? "fp64" : "fp32", linkfmt, nmu, block);
    ctx->tune_report += line;
    return RMHMC_OK;
}

extern "C" int rmhmc_set_graphs(rmhmc_ctx* ctx, int on) {
    if (!ctx) return RMHMC_EINVAL;
    ctx->use_graphs = on != 0;
    return RMHMC_OK;
}
