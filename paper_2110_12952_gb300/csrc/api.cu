// api.cu -- C ABI entry points: handle creation and validation, error
// reporting, multi-step ping-pong and host-buffer calls.  Kernels live in
// maps.cu (lambda, nu, init, scatter/gather), step.cu (compact step) and
// bb.cu (bounding-box step).
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "handle.h"

namespace fr {

static thread_local std::string g_err;

void set_error(int code, const std::string &msg)
{
    (void)code;
    g_err = msg;
}

void clear_error() { g_err.clear(); }

int cuda_fail(cudaError_t e, const char *what)
{
    set_error(FR_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
    if (e == cudaErrorMemoryAllocation) return FR_ENOMEM;
    return FR_ECUDA;
}

static int fail(int code, const std::string &msg)
{
    set_error(code, msg);
    return code;
}

static bool mul_ok(int64_t a, int64_t b, int64_t limit, int64_t *out)
{
    if (a != 0 && b > limit / a) return false;
    *out = a * b;
    return true;
}

int launch_copy_normalise(const uint8_t *in, uint8_t *out, int64_t n, int num_sms, cudaStream_t st);
int preload_copy_kernel();

int ensure_status(fractal *f)
{
    if (f->status) return FR_OK;
    FR_CUDA(cudaMalloc(&f->status, sizeof(int)));
    FR_CUDA(cudaMemset(f->status, 0, sizeof(int)));
    return FR_OK;
}

// Reads and clears the device status word (call after the work finished).
int take_status(fractal *f)
{
    if (!f->status) return FR_OK;
    int v = 0;
    FR_CUDA(cudaMemcpy(&v, f->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (v != 0) {
        FR_CUDA(cudaMemset(f->status, 0, sizeof(int)));
        set_error(v, "a bounded device-side wait gave up; the results of that call are invalid");
        return v;
    }
    return FR_OK;
}

}  // namespace fr

using namespace fr;

extern "C" const char *fractal_last_error(void) { return g_err.c_str(); }

extern "C" const char *fractal_version(void) { return "compact-fractal-ca 0.1 (sm_103a)"; }

extern "C" int fractal_create(int k, int s, int r, int dim, const int32_t *offsets,
                              fractal_t **out)
{
    g_err.clear();
    if (!out) return fail(FR_EINVAL, "fractal_create: out is NULL");
    *out = nullptr;
    if (!offsets) return fail(FR_EINVAL, "fractal_create: offsets is NULL");
    if (dim != 2 && dim != 3) return fail(FR_EINVAL, "fractal_create: dim must be 2 or 3");
    if (s < 2 || s > 16) return fail(FR_EINVAL, "fractal_create: s must be in [2,16]");
    if (r < 0) return fail(FR_EINVAL, "fractal_create: r must be >= 0");
    int sd = 1;
    for (int i = 0; i < dim; ++i) sd *= s;
    if (sd > kMaxSD) return fail(FR_EINVAL, "fractal_create: s^dim must be <= 256");
    if (k < 1 || k > sd) return fail(FR_EINVAL, "fractal_create: k must be in [1, s^dim]");
    std::vector<int> seen(sd, -1);
    for (int j = 0; j < k; ++j) {
        int t = 0, m = 1;
        for (int i = 0; i < dim; ++i) {
            int v = offsets[j * dim + i];
            if (v < 0 || v >= s)
                return fail(FR_EINVAL, "fractal_create: offset component outside [0,s)");
            t += v * m;
            m *= s;
        }
        if (seen[t] >= 0) return fail(FR_EINVAL, "fractal_create: duplicate offset rows");
        seen[t] = j;
    }
    int64_t cells = 1, side = 1;
    for (int i = 0; i < r; ++i) {
        if (!mul_ok(cells, k, (int64_t)1 << 62, &cells))
            return fail(FR_EOVERFLOW, "fractal_create: k^r >= 2^62");
        if (!mul_ok(side, s, ((int64_t)1 << 31) - 1, &side))
            return fail(FR_EOVERFLOW, "fractal_create: s^r >= 2^31");
    }
    int64_t box = 1;
    for (int i = 0; i < dim; ++i)
        if (!mul_ok(box, side, INT64_MAX, &box)) { box = -1; break; }

    fractal *f = new (std::nothrow) fractal();
    if (!f) return fail(FR_ENOMEM, "fractal_create: out of host memory");
    f->k = k; f->s = s; f->r = r; f->dim = dim;
    f->offsets.assign(offsets, offsets + (size_t)k * dim);
    f->cells = cells;
    f->side = side;
    f->box_cells = box;
    FracDev &D = f->dev;
    memset(&D, 0, sizeof(D));
    D.k = k; D.s = s; D.r = r; D.dim = dim; D.sd = sd;
    D.sdiv = make_div((uint32_t)s);
    D.kdiv = make_div((uint32_t)(k >= 2 ? k : 2));
    for (int t = 0; t < kMaxSD; ++t) D.hinv[t] = -1;
    for (int t = 0; t < sd; ++t) D.hinv[t] = (int16_t)seen[t];
    for (int j = 0; j < k; ++j)
        for (int i = 0; i < dim; ++i) D.off[j][i] = (int8_t)offsets[j * dim + i];
    cudaError_t e = cudaGetDevice(&f->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&f->num_sms, cudaDevAttrMultiProcessorCount, f->device);
    if (e != cudaSuccess) {
        delete f;
        return cuda_fail(e, "fractal_create: no usable CUDA device");
    }
    f->tile_levels_user = cached_tile_levels(f, &f->stages_user);
    *out = f;
    return FR_OK;
}

extern "C" int fractal_create_mixed(int s, int r, int dim, const int32_t *ks, const int32_t *offsets,
                                    fractal_t **out)
{
    g_err.clear();
    if (!out) return fail(FR_EINVAL, "fractal_create_mixed: out is NULL");
    *out = nullptr;
    if (!offsets || (!ks && r > 0)) return fail(FR_EINVAL, "fractal_create_mixed: NULL table");
    if (dim != 2 && dim != 3) return fail(FR_EINVAL, "fractal_create_mixed: dim must be 2 or 3");
    if (s < 2 || s > 16) return fail(FR_EINVAL, "fractal_create_mixed: s must be in [2,16]");
    if (r < 1 || r > kMaxR) return fail(FR_EINVAL, "fractal_create_mixed: r must be in [1, 62]");
    int sd = 1;
    for (int i = 0; i < dim; ++i) sd *= s;
    if (sd > kMaxSD) return fail(FR_EINVAL, "fractal_create_mixed: s^dim must be <= 256");
    std::vector<std::vector<int16_t>> hinv(r, std::vector<int16_t>(kMaxSD, -1));
    std::vector<int64_t> first(r);
    int64_t rows = 0, cells = 1, side = 1;
    for (int mu = 0; mu < r; ++mu) {
        const int k = ks[mu];
        if (k < 1 || k > sd) return fail(FR_EINVAL, "fractal_create_mixed: every k must be in [1, s^dim]");
        first[mu] = rows;
        for (int j = 0; j < k; ++j) {
            int t = 0, m = 1;
            for (int i = 0; i < dim; ++i) {
                const int v = offsets[(rows + j) * dim + i];
                if (v < 0 || v >= s) return fail(FR_EINVAL, "fractal_create_mixed: offset component outside [0,s)");
                t += v * m;
                m *= s;
            }
            if (hinv[mu][t] >= 0) return fail(FR_EINVAL, "fractal_create_mixed: duplicate offset rows in a level");
            hinv[mu][t] = (int16_t)j;
        }
        rows += k;
        if (!mul_ok(cells, k, (int64_t)1 << 62, &cells))
            return fail(FR_EOVERFLOW, "fractal_create_mixed: the cell count reaches 2^62");
        if (!mul_ok(side, s, ((int64_t)1 << 31) - 1, &side))
            return fail(FR_EOVERFLOW, "fractal_create_mixed: s^r >= 2^31");
    }
    int64_t box = 1;
    for (int i = 0; i < dim; ++i)
        if (!mul_ok(box, side, INT64_MAX, &box)) { box = -1; break; }
    fractal *f = new (std::nothrow) fractal();
    if (!f) return fail(FR_ENOMEM, "fractal_create_mixed: out of host memory");
    f->k = ks[0]; f->s = s; f->r = r; f->dim = dim;
    f->offsets.assign(offsets, offsets + (size_t)rows * dim);
    f->cells = cells;
    f->side = side;
    f->box_cells = box;
    f->mixed = true;
    f->lev_k.assign(ks, ks + r);
    f->lev_first = first;
    f->lev_hinv = hinv;
    FracDev &D = f->dev;
    memset(&D, 0, sizeof(D));
    D.k = ks[0]; D.s = s; D.r = r; D.dim = dim; D.sd = sd;
    D.sdiv = make_div((uint32_t)s);
    D.kdiv = make_div((uint32_t)(ks[0] >= 2 ? ks[0] : 2));
    for (int t = 0; t < kMaxSD; ++t) D.hinv[t] = hinv[0][t];
    std::vector<MixLevel> lv(r);
    for (int mu = 0; mu < r; ++mu) {
        memset(&lv[mu], 0, sizeof(MixLevel));
        lv[mu].k = ks[mu];
        lv[mu].kdiv = make_div((uint32_t)(ks[mu] >= 2 ? ks[mu] : 2));
        for (int t = 0; t < kMaxSD; ++t) lv[mu].hinv[t] = hinv[mu][t];
        for (int j = 0; j < ks[mu]; ++j)
            for (int i = 0; i < dim; ++i) lv[mu].off[j][i] = (int8_t)offsets[(first[mu] + j) * dim + i];
    }
    for (int j = 0; j < ks[0]; ++j)
        for (int i = 0; i < dim; ++i) D.off[j][i] = lv[0].off[j][i];
    cudaError_t e = cudaGetDevice(&f->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&f->num_sms, cudaDevAttrMultiProcessorCount, f->device);
    if (e == cudaSuccess) e = cudaMalloc(&f->d_mix, sizeof(MixLevel) * (size_t)r);
    if (e == cudaSuccess) e = cudaMemcpy(f->d_mix, lv.data(), sizeof(MixLevel) * (size_t)r, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(f->d_mix);
        delete f;
        return cuda_fail(e, "fractal_create_mixed: no usable CUDA device");
    }
    D.mix = f->d_mix;
    f->tile_levels_user = cached_tile_levels(f, &f->stages_user);
    *out = f;
    return FR_OK;
}

static void free_pipe(HostPipe &p);

extern "C" int fractal_destroy(fractal_t *f)
{
    g_err.clear();
    if (!f) return FR_OK;
    cudaDeviceSynchronize();
    free_step_plan(f->plan);
    free_tb_plan(f->tb);
    fr_paper_aux_free(f);
    free_bb_plan(f->bb);
    cudaFree(f->scratch);
    cudaFree(f->b3_state[0]);
    cudaFree(f->b3_state[1]);
    cudaFree(f->bb_scratch);
    cudaFree(f->host_io[0]);
    cudaFree(f->host_io[1]);
    cudaFree(f->status);
    cudaFree(f->d_mix);
    free_pipe(f->pipe);
    delete f;
    return FR_OK;
}

extern "C" int fractal_info(const fractal_t *f, int64_t *cells, int64_t *side)
{
    g_err.clear();
    if (!f) return fail(FR_EINVAL, "fractal_info: handle is NULL");
    if (cells) *cells = f->cells;
    if (side) *side = f->side;
    return FR_OK;
}

extern "C" int fractal_set_tile_levels(fractal_t *f, int levels)
{
    g_err.clear();
    if (!f) return fail(FR_EINVAL, "fractal_set_tile_levels: handle is NULL");
    if (levels < -1 || levels > f->r)
        return fail(FR_EINVAL, "fractal_set_tile_levels: levels must be -1 or in [0, r]");
    if (levels != f->tile_levels_user && f->server_refs.load() > 0)
        return fail(FR_EBUSY, "fractal_set_tile_levels: a server still holds requests on this handle");
    if (levels != f->tile_levels_user) {
        f->tile_levels_user = levels;
        cudaDeviceSynchronize();
        free_step_plan(f->plan);
    }
    return FR_OK;
}

extern "C" int fractal_set_pipeline_stages(fractal_t *f, int stages)
{
    g_err.clear();
    if (!f) return fail(FR_EINVAL, "fractal_set_pipeline_stages: handle is NULL");
    if (stages != -1 && (stages < 2 || stages > 4))
        return fail(FR_EINVAL, "fractal_set_pipeline_stages: stages must be -1 or in [2, 4]");
    if (stages != f->stages_user && f->server_refs.load() > 0)
        return fail(FR_EBUSY, "fractal_set_pipeline_stages: a server still holds requests on this handle");
    if (stages != f->stages_user) {
        f->stages_user = stages;
        cudaDeviceSynchronize();
        free_step_plan(f->plan);
    }
    return FR_OK;
}

extern "C" int fractal_get_tile_levels(const fractal_t *f, int *levels)
{
    g_err.clear();
    if (!f || !levels) return fail(FR_EINVAL, "fractal_get_tile_levels: NULL argument");
    int rc = ensure_step_plan(const_cast<fractal_t *>(f));
    if (rc) return rc;
    *levels = f->plan.L;
    return FR_OK;
}

extern "C" int fractal_plan_info(const fractal_t *f, int32_t *info, int n)
{
    g_err.clear();
    if (!f || !info) return fail(FR_EINVAL, "fractal_plan_info: NULL argument");
    if (n < 1 || n > 7) return fail(FR_EINVAL, "fractal_plan_info: n must be in [1, 7]");
    int rc = ensure_step_plan(const_cast<fractal_t *>(f));
    if (rc) return rc;
    const StepPlan &p = f->plan;
    const int32_t v[7] = {p.mode, p.L, p.block, p.grid, p.smem, p.nstage, p.per_sm};
    for (int i = 0; i < n; ++i) info[i] = v[i];
    return FR_OK;
}

static bool overlap(const void *a, const void *b, int64_t n)
{
    const uint8_t *x = (const uint8_t *)a, *y = (const uint8_t *)b;
    return x < y + n && y < x + n;
}

static int ensure_buffer(uint8_t **buf, int64_t bytes, const char *what)
{
    if (*buf) return FR_OK;
    cudaError_t e = cudaMalloc((void **)buf, (size_t)bytes);
    if (e != cudaSuccess) {
        *buf = nullptr;
        return cuda_fail(e, what);
    }
    return FR_OK;
}

// Ping-pong `steps` generations so that the last one lands in `out`: step i
// (1-based) writes `out` when steps - i is even, the scratch buffer otherwise.
template <class Launch>
static int run_generations(const uint8_t *in, uint8_t *out, uint8_t *scratch, int64_t steps,
                           Launch launch)
{
    const uint8_t *src = in;
    for (int64_t i = 1; i <= steps; ++i) {
        uint8_t *dst = ((steps - i) % 2 == 0) ? out : scratch;
        int rc = launch(src, dst);
        if (rc) return rc;
        src = dst;
    }
    return FR_OK;
}

extern "C" int fractal_step(fractal_t *f, const uint8_t *in, uint8_t *out, int64_t steps,
                            uint32_t birth, uint32_t survive, void *stream)
{
    g_err.clear();
    if (!f || !in || !out) return fail(FR_EINVAL, "fractal_step: NULL argument");
    if (steps < 0) return fail(FR_EINVAL, "fractal_step: steps < 0");
    if (overlap(in, out, f->cells)) return fail(FR_EINVAL, "fractal_step: in and out overlap");
    cudaStream_t st = (cudaStream_t)stream;
    if (steps == 0) return launch_copy_normalise(in, out, f->cells, f->num_sms, st);
    if (f->tb_gens > 0) {
        // temporal blocking: passes of up to tb_gens generations each; pass
        // i (1-based) of n writes `out` when n - i is even, else the scratch
        int rc = ensure_tb_plan(f);
        if (rc) return rc;
        const int64_t passes = (steps + f->tb_gens - 1) / f->tb_gens;
        if (passes > 1) {
            rc = ensure_buffer(&f->scratch, f->cells, "fractal_step: scratch allocation");
            if (rc) return rc;
        }
        const uint8_t *src = in;
        int64_t left = steps;
        for (int64_t i = 1; i <= passes; ++i) {
            uint8_t *dst = ((passes - i) % 2 == 0) ? out : f->scratch;
            const int g = (int)std::min<int64_t>(left, f->tb_gens);
            rc = launch_tb_once(f, src, dst, g, birth, survive, st);
            if (rc) return rc;
            left -= g;
            src = dst;
        }
        return FR_OK;
    }
    int rc = ensure_step_plan(f);
    if (rc) return rc;
    if (steps > 1 && bit3_plan(f)) return launch_bit3_generations(f, in, out, steps, birth, survive, st);
    if (steps > 1) {
        rc = ensure_buffer(&f->scratch, f->cells, "fractal_step: scratch allocation");
        if (rc) return rc;
    }
    return run_generations(in, out, f->scratch, steps, [&](const uint8_t *a, uint8_t *b) {
        return launch_step_once(f, a, b, birth, survive, st);
    });
}

extern "C" int fractal_set_temporal_blocking(fractal_t *f, int generations, int tile_levels)
{
    g_err.clear();
    if (!f) return fail(FR_EINVAL, "fractal_set_temporal_blocking: handle is NULL");
    if (generations < 0 || generations > kTbMaxGenerations)
        return fail(FR_EINVAL, "fractal_set_temporal_blocking: generations must be in [0, 9]");
    if (tile_levels != -1 && (tile_levels < 2 || tile_levels > f->r))
        return fail(FR_EINVAL, "fractal_set_temporal_blocking: tile_levels must be -1 or in [2, r]");
    const int old_g = f->tb_gens, old_l = f->tb_levels_user;
    f->tb_gens = generations;
    f->tb_levels_user = tile_levels;
    if (generations > 0) {
        if (tile_levels != old_l) {
            cudaDeviceSynchronize();
            free_tb_plan(f->tb);
        }
        const int rc = ensure_tb_plan(f);
        if (rc) {
            f->tb_gens = old_g;
            f->tb_levels_user = old_l;
            return rc;
        }
    }
    return FR_OK;
}

extern "C" int fractal_bb_step(fractal_t *f, const uint8_t *in, uint8_t *out, int64_t steps,
                               uint32_t birth, uint32_t survive, void *stream)
{
    g_err.clear();
    if (!f || !in || !out) return fail(FR_EINVAL, "fractal_bb_step: NULL argument");
    if (steps < 0) return fail(FR_EINVAL, "fractal_bb_step: steps < 0");
    if (f->box_cells < 0) return fail(FR_EOVERFLOW, "fractal_bb_step: n^dim overflows");
    if (overlap(in, out, f->box_cells))
        return fail(FR_EINVAL, "fractal_bb_step: in and out overlap");
    cudaStream_t st = (cudaStream_t)stream;
    int rc = ensure_bb_plan(f);
    if (rc) return rc;
    if (steps == 0) {
        // zero generations: the masked, normalised box (no births; every
        // live member survives whatever its count)
        return launch_bb_once(f, in, out, 0u, 0xffffffffu, st);
    }
    if (steps > 1) {
        rc = ensure_buffer(&f->bb_scratch, f->box_cells, "fractal_bb_step: scratch allocation");
        if (rc) return rc;
    }
    return run_generations(in, out, f->bb_scratch, steps, [&](const uint8_t *a, uint8_t *b) {
        return launch_bb_once(f, a, b, birth, survive, st);
    });
}

static void free_pipe(HostPipe &p)
{
    if (p.s_h2d) cudaStreamDestroy(p.s_h2d);
    if (p.s_comp) cudaStreamDestroy(p.s_comp);
    if (p.s_d2h) cudaStreamDestroy(p.s_d2h);
    for (cudaEvent_t e : p.ev_in) cudaEventDestroy(e);
    for (cudaEvent_t e : p.ev_out) cudaEventDestroy(e);
    if (p.ev_start) cudaEventDestroy(p.ev_start);
    if (p.ev_done) cudaEventDestroy(p.ev_done);
    p = HostPipe();
}

// Chunks of about kPipeChunkBytes (at most 64) and their schedule, from the
// neighbour-tile table of the current step plan.
constexpr int64_t kPipeChunkBytes = (int64_t)32 << 20;

static int ensure_pipe(fractal *f)
{
    HostPipe &p = f->pipe;
    if (p.L == f->plan.L && p.NT == f->plan.NT && !p.bounds.empty()) return FR_OK;
    free_pipe(p);
    const int64_t NT = f->plan.NT;
    const int C = (int)std::max<int64_t>(1, std::min<int64_t>({64, NT, f->cells / kPipeChunkBytes}));
    p.bounds.resize(C + 1);
    for (int c = 0; c <= C; ++c) p.bounds[c] = NT * c / C;
    std::vector<int32_t> nbr((size_t)(NT * f->plan.nbrw));
    FR_CUDA(cudaMemcpy(nbr.data(), f->plan.nbr, nbr.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
    p.need.assign(C, 0);
    int c = 0;
    for (int64_t T = 0; T < NT; ++T) {
        while (T >= p.bounds[c + 1]) ++c;
        int64_t far = T;
        for (int d = 0; d < f->plan.nbrw; ++d) far = std::max<int64_t>(far, nbr[(size_t)(T * f->plan.nbrw + d)]);
        const int fc = (int)(std::upper_bound(p.bounds.begin(), p.bounds.end(), far) - p.bounds.begin()) - 1;
        p.need[c] = std::max(p.need[c], fc);
    }
    p.order.resize(C);
    for (int i = 0; i < C; ++i) p.order[i] = i;
    std::stable_sort(p.order.begin(), p.order.end(), [&](int a, int b) { return p.need[a] < p.need[b]; });
    FR_CUDA(cudaStreamCreateWithFlags(&p.s_h2d, cudaStreamNonBlocking));
    FR_CUDA(cudaStreamCreateWithFlags(&p.s_comp, cudaStreamNonBlocking));
    FR_CUDA(cudaStreamCreateWithFlags(&p.s_d2h, cudaStreamNonBlocking));
    p.ev_in.assign(C, nullptr);
    p.ev_out.assign(C, nullptr);
    for (int i = 0; i < C; ++i) {
        FR_CUDA(cudaEventCreateWithFlags(&p.ev_in[i], cudaEventDisableTiming));
        FR_CUDA(cudaEventCreateWithFlags(&p.ev_out[i], cudaEventDisableTiming));
    }
    FR_CUDA(cudaEventCreateWithFlags(&p.ev_start, cudaEventDisableTiming));
    FR_CUDA(cudaEventCreateWithFlags(&p.ev_done, cudaEventDisableTiming));
    p.L = f->plan.L;
    p.NT = NT;
    return FR_OK;
}

// One generation from host memory to host memory, pipelined over chunks of
// tiles: the host-to-device and device-to-host copies run at the same time
// (the link carries both directions at once), each chunk computed as soon
// as its inputs have landed.
static int run_host_pipelined(fractal *f, const uint8_t *host_in, uint8_t *host_out, uint32_t birth,
                              uint32_t survive, cudaStream_t st)
{
    int rc = ensure_pipe(f);
    if (rc) return rc;
    HostPipe &p = f->pipe;
    const int64_t KL = f->plan.KL;
    const int C = (int)p.need.size();
    uint8_t *din = f->host_io[0], *dout = f->host_io[1];
    FR_CUDA(cudaEventRecord(p.ev_start, st));
    FR_CUDA(cudaStreamWaitEvent(p.s_h2d, p.ev_start, 0));
    FR_CUDA(cudaStreamWaitEvent(p.s_comp, p.ev_start, 0));
    FR_CUDA(cudaStreamWaitEvent(p.s_d2h, p.ev_start, 0));
    for (int j = 0; j < C; ++j) {
        const int64_t b0 = p.bounds[j] * KL, b1 = p.bounds[j + 1] * KL;
        FR_CUDA(cudaMemcpyAsync(din + b0, host_in + b0, (size_t)(b1 - b0), cudaMemcpyHostToDevice, p.s_h2d));
        FR_CUDA(cudaEventRecord(p.ev_in[j], p.s_h2d));
    }
    for (int i = 0; i < C; ++i) {
        const int c = p.order[i];
        FR_CUDA(cudaStreamWaitEvent(p.s_comp, p.ev_in[p.need[c]], 0));
        rc = launch_step_range(f, din, dout, p.bounds[c], p.bounds[c + 1], birth, survive, p.s_comp);
        if (rc) return rc;
        FR_CUDA(cudaEventRecord(p.ev_out[c], p.s_comp));
        FR_CUDA(cudaStreamWaitEvent(p.s_d2h, p.ev_out[c], 0));
        const int64_t b0 = p.bounds[c] * KL, b1 = p.bounds[c + 1] * KL;
        FR_CUDA(cudaMemcpyAsync(host_out + b0, dout + b0, (size_t)(b1 - b0), cudaMemcpyDeviceToHost, p.s_d2h));
    }
    FR_CUDA(cudaEventRecord(p.ev_done, p.s_d2h));
    FR_CUDA(cudaStreamWaitEvent(st, p.ev_done, 0));
    return FR_OK;
}

extern "C" int fractal_run_host(fractal_t *f, const uint8_t *host_in, uint8_t *host_out,
                                int64_t steps, uint32_t birth, uint32_t survive, void *stream)
{
    g_err.clear();
    if (!f || !host_in || !host_out) return fail(FR_EINVAL, "fractal_run_host: NULL argument");
    if (steps < 0) return fail(FR_EINVAL, "fractal_run_host: steps < 0");
    cudaStream_t st = (cudaStream_t)stream;
    int rc = ensure_buffer(&f->host_io[0], f->cells, "fractal_run_host: device buffer");
    if (!rc) rc = ensure_buffer(&f->host_io[1], f->cells, "fractal_run_host: device buffer");
    if (rc) return rc;
    if (steps == 1 && f->tb_gens == 0) {
        rc = ensure_step_plan(f);
        if (rc) return rc;
        rc = run_host_pipelined(f, host_in, host_out, birth, survive, st);
        if (rc) return rc;
        FR_CUDA(cudaStreamSynchronize(st));
        return take_status(f);
    }
    FR_CUDA(cudaMemcpyAsync(f->host_io[0], host_in, (size_t)f->cells, cudaMemcpyHostToDevice, st));
    rc = fractal_step(f, f->host_io[0], f->host_io[1], steps, birth, survive, stream);
    if (rc) return rc;
    FR_CUDA(cudaMemcpyAsync(host_out, f->host_io[1], (size_t)f->cells, cudaMemcpyDeviceToHost, st));
    FR_CUDA(cudaStreamSynchronize(st));
    return take_status(f);
}

extern "C" int fractal_sync(void *stream)
{
    g_err.clear();
    FR_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    FR_CUDA(cudaGetLastError());
    return FR_OK;
}

extern "C" int fractal_check(fractal_t *f)
{
    g_err.clear();
    if (!f) return fail(FR_EINVAL, "fractal_check: handle is NULL");
    FR_CUDA(cudaDeviceSynchronize());
    return take_status(f);
}

extern "C" int fractal_test_arm_timeout(fractal_t *f, uint32_t extra_bytes, uint32_t wait_tries)
{
    g_err.clear();
    if (!f) return fail(FR_EINVAL, "fractal_test_arm_timeout: handle is NULL");
    if (extra_bytes < 1 || extra_bytes > 4096 || wait_tries < 1 || wait_tries > (1u << 20))
        return fail(FR_EINVAL, "fractal_test_arm_timeout: extra_bytes must be in [1, 4096] and "
                               "wait_tries in [1, 2^20]");
    f->test_extra_tx = extra_bytes;
    f->test_wait_limit = wait_tries;
    return FR_OK;
}

extern "C" int fractal_autotune(fractal_t *f, const uint8_t *in, uint8_t *out, uint32_t birth,
                                uint32_t survive, void *stream, int *levels)
{
    g_err.clear();
    if (!f || !in || !out) return fail(FR_EINVAL, "fractal_autotune: NULL argument");
    if (overlap(in, out, f->cells)) return fail(FR_EINVAL, "fractal_autotune: in and out overlap");
    if (f->server_refs.load() > 0)
        return fail(FR_EBUSY, "fractal_autotune: a server still holds requests on this handle");
    return autotune_step(f, in, out, birth, survive, (cudaStream_t)stream, levels);
}
