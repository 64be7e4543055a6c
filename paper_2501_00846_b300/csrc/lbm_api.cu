// C ABI (include/lbm.h): context management, validation, buffer ownership and dispatch.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>

#include <cuda_runtime.h>

#include "lbm.h"
#include "tslb_internal.h"

namespace {

thread_local char g_last_error[512] = "";

lbm_status fail(lbm_status s, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof g_last_error, fmt, ap);
    va_end(ap);
    return s;
}

#define CUDA_TRY(call)                                                                           \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess)                                                                   \
            return fail(LBM_ERR_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),     \
                        __FILE__, __LINE__);                                                     \
    } while (0)

}  // namespace

namespace tslb {
// Record a failure message for lbm_last_error() from another translation unit.
void set_last_error(const char *msg) { snprintf(g_last_error, sizeof g_last_error, "%s", msg); }

// Grid and FP32 kernel constants of a parameter set (beta = 12 sigma / W, kappa = 3 sigma W / 2,
// kappa_AC = 4 D / W; Section "Phase-field model").
void params_to_consts(const lbm_params &p, Grid &G, Phys &P)
{
    G.nx = p.nx;
    G.ny = p.ny;
    G.nz = p.nz;
    G.nxy = p.nx * p.ny;
    G.N = p.nx * p.ny * p.nz;
    G.wall = p.wall_z;
    P.rho_g = (float)p.rho_g;
    P.drho = (float)(p.rho_l - p.rho_g);
    P.mu_g = (float)p.mu_g;
    P.dmu = (float)(p.mu_l - p.mu_g);
    P.beta4 = (float)(4.0 * 12.0 * p.sigma / p.width);
    P.kappa = (float)(1.5 * p.sigma * p.width);
    P.mob = (float)p.mobility;
    P.kac = (float)(4.0 * p.mobility / p.width);
    for (int a = 0; a < 3; ++a) {
        P.grav[a] = (float)p.gravity[a];
        P.body[a] = (float)p.body[a];
    }
    P.rho_ref = (float)p.rho_ref;
}
}  // namespace tslb

struct lbm_ctx {
    lbm_params prm;
    tslb::Grid G;
    tslb::Phys P;
    float *g[2] = {nullptr, nullptr};  // populations: FP32 g, 16-bit h (storage 1 / 2), or the 10 moment
                                       // arrays of LBM_MOM
    float *pst[2] = {nullptr, nullptr};  // stored p* of the 16-bit formats (N floats)
    float *phi[2] = {nullptr, nullptr};
    float *u[2] = {nullptr, nullptr};
    float *flux = nullptr;            // 3N Allen–Cahn flux W of the current state (paths 0, 1)
    bool w_valid = false;             // flux holds W(phi^n, ubar^n) of the current state
    double *partials = nullptr;       // observables pass-1 records
    double *result = nullptr;         // observables pass-2 record (device)
    double *h_result = nullptr;       // pinned host copy
    int nblocks = 0;
    int cur = 0;                      // index of the buffers holding S^n
    long long step = 0;
    bool initialized = false;
    cudaStream_t stream = nullptr;
    int path = 0;
    int split = 0;
    int storage = LBM_FP32;
    int advect = 0;                   // 1: literal advection u . grad(phi) (path 1)
};

namespace {

void free_ctx(lbm_ctx *c)
{
    if (!c) return;
    for (int b = 0; b < 2; ++b) {
        cudaFree(c->g[b]);
        cudaFree(c->pst[b]);
        cudaFree(c->phi[b]);
        cudaFree(c->u[b]);
    }
    cudaFree(c->flux);
    cudaFree(c->partials);
    cudaFree(c->result);
    if (c->h_result) cudaFreeHost(c->h_result);
    delete c;
}

lbm_status validate(const lbm_params *p)
{
    if (!p) return fail(LBM_ERR_ARG, "params is NULL");
    if (p->struct_size != sizeof(lbm_params))
        return fail(LBM_ERR_ARG, "params.struct_size = %zu, expected %zu", p->struct_size, sizeof(lbm_params));
    if (p->nx < 4 || p->ny < 4 || p->nz < 4) return fail(LBM_ERR_ARG, "nx, ny, nz must be >= 4");
    const long long n = (long long)p->nx * p->ny * p->nz;
    if (n >= (1LL << 31)) return fail(LBM_ERR_ARG, "nx*ny*nz must be < 2^31");
    if (p->ny > 65535 || p->nz > 65535) return fail(LBM_ERR_ARG, "ny, nz must be <= 65535");
    if (p->wall_z != 0 && p->wall_z != 1) return fail(LBM_ERR_ARG, "wall_z must be 0 or 1");
    if (!(p->rho_l > 0) || !(p->rho_g > 0)) return fail(LBM_ERR_ARG, "densities must be > 0");
    if (!(p->mu_l > 0) || !(p->mu_g > 0)) return fail(LBM_ERR_ARG, "viscosities must be > 0");
    if (!(p->width > 0)) return fail(LBM_ERR_ARG, "interface width must be > 0");
    if (!(p->sigma >= 0) || !isfinite(p->sigma)) return fail(LBM_ERR_ARG, "sigma must be finite and >= 0");
    if (!(p->mobility >= 0) || !(p->mobility * 52.0 / 9.0 < 2.0))
        return fail(LBM_ERR_ARG, "mobility must satisfy 0 <= D < 9/26 (FTCS limit)");
    for (int a = 0; a < 3; ++a)
        if (!isfinite(p->gravity[a]) || !isfinite(p->body[a])) return fail(LBM_ERR_ARG, "forces must be finite");
    if (!isfinite(p->rho_ref)) return fail(LBM_ERR_ARG, "rho_ref must be finite");
    if (p->storage < LBM_FP32 || p->storage > LBM_MOM_FP16)
        return fail(LBM_ERR_ARG, "storage must be an lbm_storage value (got %d)", p->storage);
    return LBM_OK;
}

void make_consts(lbm_ctx *c) { tslb::params_to_consts(c->prm, c->G, c->P); }

}  // namespace

namespace tslb {
lbm_status check_params(const lbm_params *p) { return validate(p); }
}  // namespace tslb

namespace {

cudaMemcpyKind kind_in(int on_device) { return on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice; }
cudaMemcpyKind kind_out(int on_device) { return on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost; }

}  // namespace

namespace tslb {
lbm_status ctx_view(lbm_ctx *ctx, CtxView *v)
{
    if (!ctx) return fail(LBM_ERR_ARG, "context is NULL");
    if (!ctx->initialized) return fail(LBM_ERR_STATE, "context is not initialised");
    const int c = ctx->cur;
    v->G = ctx->G;
    v->P = ctx->P;
    v->g = ctx->g[c];
    v->phi = ctx->phi[c];
    v->u = ctx->u[c];
    v->storage = ctx->storage;
    v->stream = ctx->stream;
    return LBM_OK;
}
void ctx_state_changed(lbm_ctx *ctx) { ctx->w_valid = false; }
}  // namespace tslb

extern "C" {

int lbm_abi_version(void) { return 1; }

const char *lbm_last_error(void) { return g_last_error; }

const char *lbm_status_string(lbm_status s)
{
    switch (s) {
    case LBM_OK: return "ok";
    case LBM_ERR_ARG: return "invalid argument";
    case LBM_ERR_OOM: return "device out of memory";
    case LBM_ERR_CUDA: return "CUDA error";
    case LBM_ERR_NONFINITE: return "non-finite values in the state";
    case LBM_ERR_TIMEOUT: return "bounded device wait expired";
    case LBM_ERR_STATE: return "call out of order";
    }
    return "unknown status";
}

lbm_status lbm_create(const lbm_params *params, lbm_ctx **out)
{
    if (!out) return fail(LBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    lbm_status st = validate(params);
    if (st != LBM_OK) return st;

    lbm_ctx *c = new (std::nothrow) lbm_ctx;
    if (!c) return fail(LBM_ERR_OOM, "host allocation failed");
    c->prm = *params;
    make_consts(c);
    const size_t N = (size_t)c->G.N;

    c->stream = (cudaStream_t)params->stream;   // NULL: the legacy default stream
    c->storage = params->storage;
    const size_t g_bytes = c->storage >= LBM_MOM    ? tslb::mom_state_bytes(c->storage, N)
                           : c->storage == LBM_FP32 ? 27 * N * sizeof(float)
                                                    : 27 * N * 2;
    const size_t pst_bytes = c->storage == LBM_BF16 || c->storage == LBM_FP16 ? N * sizeof(float) : 0;

    c->nblocks = tslb::observables_blocks(c->G);
    struct {
        void **p;
        size_t bytes;
    } allocs[] = {
        {(void **)&c->g[0], g_bytes}, {(void **)&c->g[1], g_bytes},
        {(void **)&c->pst[0], pst_bytes}, {(void **)&c->pst[1], pst_bytes},
        {(void **)&c->phi[0], N * sizeof(float)},    {(void **)&c->phi[1], N * sizeof(float)},
        {(void **)&c->u[0], 3 * N * sizeof(float)},  {(void **)&c->u[1], 3 * N * sizeof(float)},
        {(void **)&c->flux, 3 * N * sizeof(float)},
        {(void **)&c->partials, (size_t)c->nblocks * tslb::kObsFields * sizeof(double)},
        {(void **)&c->result, tslb::kObsFields * sizeof(double)},
    };
    for (auto &a : allocs) {
        if (a.bytes == 0) continue;
        cudaError_t e = cudaMalloc(a.p, a.bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            free_ctx(c);
            return fail(e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA, "cudaMalloc(%zu) failed: %s",
                        a.bytes, cudaGetErrorString(e));
        }
    }
    cudaError_t e = cudaMallocHost(&c->h_result, tslb::kObsFields * sizeof(double));
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_ctx(c);
        return fail(LBM_ERR_OOM, "cudaMallocHost failed: %s", cudaGetErrorString(e));
    }
    *out = c;
    return LBM_OK;
}

void lbm_destroy(lbm_ctx *ctx)
{
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    free_ctx(ctx);
}

long long lbm_num_nodes(const lbm_ctx *ctx) { return ctx ? (long long)ctx->G.N : 0; }
long long lbm_step_count(const lbm_ctx *ctx) { return ctx ? ctx->step : 0; }

lbm_status lbm_set_path(lbm_ctx *ctx, int path)
{
    if (!ctx) return fail(LBM_ERR_ARG, "context is NULL");
    if (path < 0 || path > 2)
        return fail(LBM_ERR_ARG, "path must be 0 (two kernels), 1 (three kernels) or 2 (one fused kernel)");
    if (path == 2 && ctx->storage != LBM_FP32)
        return fail(LBM_ERR_ARG, "16-bit and moment storage run on paths 0 and 1 only");
    if (path != 1 && ctx->advect)
        return fail(LBM_ERR_ARG, "the literal advection form runs on path 1 only");
    ctx->path = path;
    return LBM_OK;
}

lbm_status lbm_set_advection(lbm_ctx *ctx, int form)
{
    if (!ctx) return fail(LBM_ERR_ARG, "context is NULL");
    if (form != 0 && form != 1) return fail(LBM_ERR_ARG, "advection form must be 0 (flux) or 1 (literal)");
    if (form == 1 && ctx->path != 1)
        return fail(LBM_ERR_ARG, "the literal advection form runs on path 1 only (lbm_set_path(ctx, 1) first)");
    ctx->advect = form;
    return LBM_OK;
}

lbm_status lbm_set_split(lbm_ctx *ctx, int split)
{
    if (!ctx) return fail(LBM_ERR_ARG, "context is NULL");
    if (split < 0) return fail(LBM_ERR_ARG, "split must be >= 0");
    ctx->split = split;
    return LBM_OK;
}

lbm_status lbm_init_fields(lbm_ctx *ctx, const float *phi, const float *u, const float *pstar, int on_device)
{
    if (!ctx) return fail(LBM_ERR_ARG, "context is NULL");
    if (!phi || !u) return fail(LBM_ERR_ARG, "phi and u are required");
    const size_t N = (size_t)ctx->G.N;
    const int c = ctx->cur;
    CUDA_TRY(cudaMemcpyAsync(ctx->phi[c], phi, N * sizeof(float), kind_in(on_device), ctx->stream));
    CUDA_TRY(cudaMemcpyAsync(ctx->u[c], u, 3 * N * sizeof(float), kind_in(on_device), ctx->stream));
    const float *ps = nullptr;
    if (pstar) {   // stage p*0 in the idle population buffer (at least 40 N bytes)
        CUDA_TRY(cudaMemcpyAsync(ctx->g[1 - c], pstar, N * sizeof(float), kind_in(on_device), ctx->stream));
        ps = ctx->g[1 - c];
    }
    if (ctx->storage == LBM_FP32)
        CUDA_TRY(tslb::launch_init(ctx->G, ps, ctx->u[c], ctx->g[c], ctx->stream));
    else if (ctx->storage >= LBM_MOM)
        CUDA_TRY(tslb::launch_mom_init(ctx->G, ctx->storage, ps, ctx->g[c], ctx->stream));
    else
        CUDA_TRY(tslb::launch_init16(ctx->G, ctx->storage, ps, ctx->g[c], ctx->pst[c], ctx->stream));
    CUDA_TRY(tslb::launch_flux(ctx->G, ctx->P, ctx->phi[c], ctx->u[c], ctx->flux, ctx->stream));
    ctx->w_valid = true;
    if (!on_device) CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    ctx->step = 0;
    ctx->initialized = true;
    return LBM_OK;
}

lbm_status lbm_step(lbm_ctx *ctx, int nsteps)
{
    if (!ctx) return fail(LBM_ERR_ARG, "context is NULL");
    if (nsteps < 0) return fail(LBM_ERR_ARG, "nsteps must be >= 0");
    if (!ctx->initialized) return fail(LBM_ERR_STATE, "lbm_step before lbm_init_fields");
    for (int s = 0; s < nsteps; ++s) {
        const int a = ctx->cur, b = 1 - ctx->cur;
        if (ctx->path == 0 && !ctx->w_valid) {   // the flux of the current state, once
            cudaError_t e = tslb::launch_flux(ctx->G, ctx->P, ctx->phi[a], ctx->u[a], ctx->flux, ctx->stream);
            if (e != cudaSuccess) return fail(LBM_ERR_CUDA, "flux launch failed: %s", cudaGetErrorString(e));
            ctx->w_valid = true;
        }
        tslb::StepArgs args{ctx->g[a], ctx->g[b], ctx->phi[a], ctx->phi[b], ctx->u[a], ctx->u[b], ctx->flux,
                            ctx->storage, ctx->pst[a], ctx->pst[b], ctx->advect};
        cudaError_t e = ctx->path == 0   ? tslb::launch_step_split(ctx->G, ctx->P, args, ctx->split, ctx->stream)
                         : ctx->path == 2 ? tslb::launch_step_fused2(ctx->G, ctx->P, args, ctx->split, ctx->stream)
                                          : tslb::launch_step_unfused(ctx->G, ctx->P, args, ctx->stream);
        if (e != cudaSuccess) return fail(LBM_ERR_CUDA, "step launch failed: %s", cudaGetErrorString(e));
        ctx->w_valid = ctx->path != 2;   // paths 0 and 1 leave W^{n+1} in the flux buffer
        ctx->cur = b;
        ++ctx->step;
    }
    return LBM_OK;
}

lbm_status lbm_run_phase(lbm_ctx *ctx, int phase, int nrep)
{
    if (!ctx) return fail(LBM_ERR_ARG, "context is NULL");
    if (!ctx->initialized) return fail(LBM_ERR_STATE, "lbm_run_phase before lbm_init_fields");
    if (phase != 0 && phase != 1) return fail(LBM_ERR_ARG, "phase must be 0 or 1");
    if (nrep < 0) return fail(LBM_ERR_ARG, "nrep must be >= 0");
    const int a = ctx->cur, b = 1 - ctx->cur;
    if (phase == 0 && !ctx->w_valid) {
        CUDA_TRY(tslb::launch_flux(ctx->G, ctx->P, ctx->phi[a], ctx->u[a], ctx->flux, ctx->stream));
        ctx->w_valid = true;
    }
    // phase 1 writes the flux of the idle state: the current state's W is recomputed before the
    // next use
    if (phase == 1 && nrep > 0) ctx->w_valid = false;
    for (int r = 0; r < nrep; ++r) {
        cudaError_t e = phase == 0 ? tslb::launch_ac_div(ctx->G, ctx->P, ctx->phi[a], ctx->flux, ctx->phi[b], ctx->split,
                                                         ctx->stream)
                         : ctx->storage >= LBM_MOM
                             ? tslb::launch_mom(ctx->G, ctx->P, ctx->storage, ctx->g[a], ctx->u[a], ctx->phi[b],
                                                ctx->g[b], ctx->u[b], ctx->flux, ctx->split, ctx->stream)
                         : ctx->storage != LBM_FP32
                             ? tslb::launch_lbm16(ctx->G, ctx->P, ctx->storage, ctx->g[a], ctx->pst[a], ctx->phi[b],
                                                  ctx->u[a], ctx->g[b], ctx->pst[b], ctx->u[b], ctx->flux, ctx->split,
                                                  ctx->stream)
                             : tslb::launch_lbm(ctx->G, ctx->P, 0, ctx->g[a], nullptr, ctx->phi[b], ctx->u[a],
                                                ctx->g[b], nullptr, ctx->u[b], ctx->flux, ctx->stream);
        if (e != cudaSuccess) return fail(LBM_ERR_CUDA, "phase launch failed: %s", cudaGetErrorString(e));
    }
    return LBM_OK;
}

lbm_status lbm_synchronize(lbm_ctx *ctx)
{
    if (!ctx) return fail(LBM_ERR_ARG, "context is NULL");
    CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return LBM_OK;
}

lbm_status lbm_observables(lbm_ctx *ctx, lbm_obs *out)
{
    if (!ctx) return fail(LBM_ERR_ARG, "context is NULL");
    if (!out) return fail(LBM_ERR_ARG, "out is NULL");
    if (!ctx->initialized) return fail(LBM_ERR_STATE, "lbm_observables before lbm_init_fields");
    const int c = ctx->cur;
    CUDA_TRY(tslb::launch_observables(ctx->G, ctx->prm.rho_l, ctx->prm.rho_g, ctx->g[c], ctx->phi[c], ctx->u[c],
                                      ctx->partials, ctx->nblocks, ctx->result, ctx->stream, ctx->storage,
                                      ctx->pst[c]));
    CUDA_TRY(cudaMemcpyAsync(ctx->h_result, ctx->result, tslb::kObsFields * sizeof(double), cudaMemcpyDeviceToHost,
                             ctx->stream));
    CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    const double *r = ctx->h_result;
    memset(out, 0, sizeof *out);
    out->step = (double)ctx->step;
    out->sum_phi = r[0];
    out->mass = r[1];
    out->sum_pstar = r[2];
    for (int a = 0; a < 3; ++a) {
        out->momentum[a] = r[3 + a];
        out->centroid_liq[a] = r[6 + a] / r[0];
        out->centroid_gas[a] = r[9 + a] / r[26];
        out->vel_liq[a] = r[12 + a] / r[0];
        out->vel_gas[a] = r[15 + a] / r[26];
    }
    out->n_liq = r[19];
    out->n_gas = r[21];
    out->p_liq = r[19] > 0 ? r[18] / r[19] : NAN;
    out->p_gas = r[21] > 0 ? r[20] / r[21] : NAN;
    out->umax = r[22];
    out->phi_min = r[23];
    out->phi_max = r[24];
    out->n_nonfinite = r[25];
    if (out->n_nonfinite > 0) return fail(LBM_ERR_NONFINITE, "%.0f non-finite nodes", out->n_nonfinite);
    return LBM_OK;
}

lbm_status lbm_read_fields(lbm_ctx *ctx, float *phi, float *u, float *p, int on_device)
{
    if (!ctx) return fail(LBM_ERR_ARG, "context is NULL");
    if (!ctx->initialized) return fail(LBM_ERR_STATE, "lbm_read_fields before lbm_init_fields");
    const size_t N = (size_t)ctx->G.N;
    const int c = ctx->cur;
    if (phi) CUDA_TRY(cudaMemcpyAsync(phi, ctx->phi[c], N * sizeof(float), kind_out(on_device), ctx->stream));
    if (u) CUDA_TRY(cudaMemcpyAsync(u, ctx->u[c], 3 * N * sizeof(float), kind_out(on_device), ctx->stream));
    if (p) {   // compute p into the idle population buffer, then copy
        float *tmp = ctx->g[1 - c];
        CUDA_TRY(tslb::launch_pressure(ctx->G, ctx->P, ctx->storage, ctx->g[c], ctx->pst[c], ctx->phi[c], tmp,
                                       ctx->stream));
        CUDA_TRY(cudaMemcpyAsync(p, tmp, N * sizeof(float), kind_out(on_device), ctx->stream));
    }
    CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return LBM_OK;
}

lbm_status lbm_get_state(lbm_ctx *ctx, float *g, float *phi, float *u, int on_device)
{
    if (!ctx) return fail(LBM_ERR_ARG, "context is NULL");
    if (!ctx->initialized) return fail(LBM_ERR_STATE, "lbm_get_state before lbm_init_fields");
    const size_t N = (size_t)ctx->G.N;
    const int c = ctx->cur;
    if (g && ctx->storage == LBM_FP32) {
        CUDA_TRY(cudaMemcpyAsync(g, ctx->g[c], 27 * N * sizeof(float), kind_out(on_device), ctx->stream));
    } else if (g && ctx->storage >= LBM_MOM) {
        // g_i = w_i (g_i / w_i)(moments): straight into a device buffer, or a few directions at a time
        // through the idle moment buffer
        const int chunk = (int)(tslb::mom_state_bytes(ctx->storage, N) / (N * sizeof(float)));
        for (int i0 = 0; i0 < 27; i0 += on_device ? 27 : chunk) {
            const int ni = on_device ? 27 : (i0 + chunk <= 27 ? chunk : 27 - i0);
            float *dst = on_device ? g : ctx->g[1 - c];
            CUDA_TRY(tslb::launch_mom_expand(ctx->G, ctx->storage, ctx->g[c], ctx->u[c], i0, ni, dst, ctx->stream));
            if (!on_device)
                CUDA_TRY(cudaMemcpyAsync(g + (size_t)i0 * N, dst, ni * N * sizeof(float), cudaMemcpyDeviceToHost,
                                         ctx->stream));
        }
    } else if (g && on_device) {   // g_i = w_i (P + f^eq_i(0, u) / w_i + h_i) straight into the caller's buffer
        CUDA_TRY(tslb::launch_expand16(ctx->G, ctx->storage, ctx->g[c], ctx->pst[c], ctx->u[c], 0, 27, g,
                                       ctx->stream));
    } else if (g) {   // expand 13 directions at a time into the idle buffer (54 N bytes), then copy
        float *tmp = ctx->g[1 - c];
        for (int i0 = 0; i0 < 27; i0 += 13) {
            const int ni = i0 + 13 <= 27 ? 13 : 27 - i0;
            CUDA_TRY(tslb::launch_expand16(ctx->G, ctx->storage, ctx->g[c], ctx->pst[c], ctx->u[c], i0, ni, tmp,
                                           ctx->stream));
            CUDA_TRY(cudaMemcpyAsync(g + (size_t)i0 * N, tmp, ni * N * sizeof(float), cudaMemcpyDeviceToHost,
                                     ctx->stream));
        }
    }
    if (phi) CUDA_TRY(cudaMemcpyAsync(phi, ctx->phi[c], N * sizeof(float), kind_out(on_device), ctx->stream));
    if (u) CUDA_TRY(cudaMemcpyAsync(u, ctx->u[c], 3 * N * sizeof(float), kind_out(on_device), ctx->stream));
    CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return LBM_OK;
}

lbm_status lbm_set_state(lbm_ctx *ctx, const float *g, const float *phi, const float *u, long long step,
                         int on_device)
{
    if (!ctx) return fail(LBM_ERR_ARG, "context is NULL");
    if (!g || !phi || !u) return fail(LBM_ERR_ARG, "g, phi and u are required");
    if (step < 0) return fail(LBM_ERR_ARG, "step must be >= 0");
    const size_t N = (size_t)ctx->G.N;
    const int c = ctx->cur;
    CUDA_TRY(cudaMemcpyAsync(ctx->phi[c], phi, N * sizeof(float), kind_in(on_device), ctx->stream));
    CUDA_TRY(cudaMemcpyAsync(ctx->u[c], u, 3 * N * sizeof(float), kind_in(on_device), ctx->stream));
    if (ctx->storage == LBM_FP32) {
        CUDA_TRY(cudaMemcpyAsync(ctx->g[c], g, 27 * N * sizeof(float), kind_in(on_device), ctx->stream));
    } else if (ctx->storage >= LBM_MOM) {
        // population moments summed into an FP32 accumulator (the moment buffer itself with FP32
        // storage, else a temporary buffer; host input staged a few directions at a time in the idle
        // moment buffer), then converted to (p*, a, B) with u already in place
        float *acc = ctx->g[c];
        if (ctx->storage != LBM_MOM) {
            cudaError_t e = cudaMalloc(&acc, tslb::kMomArrays * N * sizeof(float));
            if (e != cudaSuccess) {
                cudaGetLastError();
                return fail(e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA,
                            "cudaMalloc of the projection buffer failed: %s", cudaGetErrorString(e));
            }
        }
        const int chunk = (int)(tslb::mom_state_bytes(ctx->storage, N) / (N * sizeof(float)));
        cudaError_t e = cudaMemsetAsync(acc, 0, tslb::kMomArrays * N * sizeof(float), ctx->stream);
        for (int i0 = 0; i0 < 27 && e == cudaSuccess; i0 += on_device ? 27 : chunk) {
            const int ni = on_device ? 27 : (i0 + chunk <= 27 ? chunk : 27 - i0);
            const float *src = g;
            if (!on_device) {
                e = cudaMemcpyAsync(ctx->g[1 - c], g + (size_t)i0 * N, ni * N * sizeof(float), cudaMemcpyHostToDevice,
                                    ctx->stream);
                src = ctx->g[1 - c];
            }
            if (e == cudaSuccess) e = tslb::launch_mom_project(ctx->G, src, i0, ni, acc, ctx->stream);
        }
        if (e == cudaSuccess) e = tslb::launch_mom_finish(ctx->G, ctx->storage, ctx->u[c], acc, ctx->g[c], ctx->stream);
        if (acc != ctx->g[c]) {
            const cudaError_t e2 = cudaStreamSynchronize(ctx->stream);
            cudaFree(acc);
            if (e == cudaSuccess) e = e2;
        }
        if (e != cudaSuccess) return fail(LBM_ERR_CUDA, "moment import failed: %s", cudaGetErrorString(e));
    } else {
        // P = sum g (mode 0), then h_i = g_i / w_i - P - f^eq_i(0, u) / w_i and P -= sum w_i h_i
        // (mode 1 + finish), with u already in place.  Host input is staged 13 directions at a
        // time in the idle population buffer (54 N bytes); corr uses the flux scratch.
        float *corr = ctx->flux;
        CUDA_TRY(cudaMemsetAsync(ctx->pst[c], 0, N * sizeof(float), ctx->stream));
        CUDA_TRY(cudaMemsetAsync(corr, 0, N * sizeof(float), ctx->stream));
        for (int mode = 0; mode < 2; ++mode) {
            if (on_device) {
                CUDA_TRY(tslb::launch_compress16(ctx->G, ctx->storage, g, ctx->u[c], 0, 27, mode, ctx->g[c],
                                                 ctx->pst[c], corr, ctx->stream));
                continue;
            }
            float *tmp = ctx->g[1 - c];
            for (int i0 = 0; i0 < 27; i0 += 13) {
                const int ni = i0 + 13 <= 27 ? 13 : 27 - i0;
                CUDA_TRY(cudaMemcpyAsync(tmp, g + (size_t)i0 * N, ni * N * sizeof(float), cudaMemcpyHostToDevice,
                                         ctx->stream));
                CUDA_TRY(tslb::launch_compress16(ctx->G, ctx->storage, tmp, ctx->u[c], i0, ni, mode, ctx->g[c],
                                                 ctx->pst[c], corr, ctx->stream));
            }
        }
        CUDA_TRY(tslb::launch_finish16(ctx->G, corr, ctx->pst[c], ctx->stream));
    }
    CUDA_TRY(tslb::launch_flux(ctx->G, ctx->P, ctx->phi[c], ctx->u[c], ctx->flux, ctx->stream));
    ctx->w_valid = true;
    CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    ctx->step = step;
    ctx->initialized = true;
    return LBM_OK;
}

}  // extern "C"
