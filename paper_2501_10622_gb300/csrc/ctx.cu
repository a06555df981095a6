// ctx.cu -- the public C ABI of libcwthf.so: context lifetime, argument
// checks, and the order of the stages (Sec. 2 step list of the paper).
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "internal.cuh"

namespace cwthf {

bool fft_size_supported(int ng);

// An NVTX range around the host-side enqueue of one stage (profilers show it
// on the CPU timeline and project it onto the kernels it launched).
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};

constexpr unsigned kCreateFlags = CWTHF_CREATE_UNBIND;

int check_ng(int ng) {
    if (ng < CWTHF_MIN_NG || ng > CWTHF_MAX_NG || ng % 2) return CWTHF_E_UNSUPPORTED_SIZE;
    return fft_size_supported(ng) ? CWTHF_OK : CWTHF_E_UNSUPPORTED_SIZE;
}

int cuda_status(cudaError_t e) { return e == cudaSuccess ? CWTHF_OK : CWTHF_E_CUDA; }

namespace {

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

struct Sizes {
    int64_t cells, nwords, slots, keys, np;
    size_t scan_words;
};

Sizes sizes_for(int max_ng, int64_t max_np) {
    Sizes z;
    z.cells = int64_t(max_ng) * max_ng * max_ng;
    z.nwords = (z.cells + 31) / 32;
    z.slots = z.cells / 8 + 8;  // at most one maximum per 2x2x2 block of cells
    z.keys = deposit_geom(max_ng).ntiles * kDepClasses;
    z.np = std::max<int64_t>(max_np, 1);
    int64_t scan_n = std::max(z.keys, std::max(z.nwords, z.slots));
    z.scan_words = scan_tmp_words(scan_n) + 2;
    return z;
}

// One table slot: the largest twiddle table of a grid size up to max_ng (3 ng
// floats, plus for Bluestein passes chirps, transformed chirps and inner
// twiddles of at most 2.25 times the pass length + 64: below 19.5 ng + 512).
size_t table_slot_floats(int max_ng) { return 20 * size_t(max_ng) + 512; }

// The allocation plan: (pointer slot, bytes).  One list drives both
// cwthf_create and cwthf_workspace_bytes.
template <class F>
void for_each_buffer(cwthf_ctx* c, int max_ng, int64_t max_np, int max_scales, unsigned flags, F&& f) {
    Sizes z = sizes_for(max_ng, max_np);
    f(reinterpret_cast<void**>(&c->d_status), sizeof(int) * 4);
    f(reinterpret_cast<void**>(&c->dep_count), size_t(z.keys + 1) * 4);
    f(reinterpret_cast<void**>(&c->dep_off), size_t(z.keys + 2) * 4);
    f(reinterpret_cast<void**>(&c->dep_cursor), size_t(z.keys + 1) * 4);
    f(reinterpret_cast<void**>(&c->dep_rec), size_t(z.np) * 8);
    f(reinterpret_cast<void**>(&c->dep_mq), size_t(z.np) * 4);
    f(reinterpret_cast<void**>(&c->part_rec), size_t(z.np) * 4);
    f(reinterpret_cast<void**>(&c->d_mtot), 16);
    f(reinterpret_cast<void**>(&c->n_seeds), 16);
    f(reinterpret_cast<void**>(&c->spec), spec_bytes(max_ng));
    if (max_scales > 1) f(reinterpret_cast<void**>(&c->spec2), spec_bytes(max_ng));
    f(reinterpret_cast<void**>(&c->seed_bits), size_t(z.nwords + 1) * 4);
    f(reinterpret_cast<void**>(&c->seed_prefix), size_t(z.nwords + 2) * 4);
    f(reinterpret_cast<void**>(&c->seed_cells), size_t(z.cells) * 4);
    f(reinterpret_cast<void**>(&c->seed_list), size_t(z.slots) * 4);
    f(reinterpret_cast<void**>(&c->acc), size_t(z.slots) * sizeof(HaloAcc));
    f(reinterpret_cast<void**>(&c->keep_off), size_t(z.slots + 2) * 4);
    f(reinterpret_cast<void**>(&c->slot_halo), size_t(z.slots) * 4 * size_t(std::max(max_scales, 1)));
    // record slots of every scale (scale-major), then (several scales) the
    // records' halo ids in groups of 2 or 4k scales; one scale's ids replace
    // its slots in place
    const size_t ms = size_t(std::max(max_scales, 1));
    const size_t groups = ms == 1 ? 0 : (ms == 2 ? 2 : (ms + 3) & ~size_t(3));
    f(reinterpret_cast<void**>(&c->part_slot), (size_t(z.np) * ms + 4) * 4 + size_t(z.np) * 4 * groups);
    f(reinterpret_cast<void**>(&c->jump_changed), sizeof(int) * kJumpWords);
    f(reinterpret_cast<void**>(&c->dep_parts), size_t(tile_parts_cap(z.np)) * 8);
    f(reinterpret_cast<void**>(&c->dep_nparts), 16);
    if (flags & CWTHF_CREATE_UNBIND) {  // self-boundness check scratch (36 bytes per particle + 24 per group)
        f(reinterpret_cast<void**>(&c->ub_off), size_t(z.slots + 2) * 4);
        f(reinterpret_cast<void**>(&c->ub_cur), size_t(z.slots + 1) * 4);
        f(reinterpret_cast<void**>(&c->ub_mem), size_t(z.np) * 4);
        f(reinterpret_cast<void**>(&c->ub_key), size_t(z.np) * 16);
        f(reinterpret_cast<void**>(&c->ub_val), size_t(z.np) * 8);
        f(reinterpret_cast<void**>(&c->ub_grp), size_t(z.np) * 4);
        f(reinterpret_cast<void**>(&c->ub_out), size_t(z.np) * 4);
        f(reinterpret_cast<void**>(&c->ub_nk), size_t(z.slots + 1) * 8);
        f(reinterpret_cast<void**>(&c->ub_it), size_t(z.slots + 1) * 4);
        f(reinterpret_cast<void**>(&c->ub_keep), size_t(z.slots + 2) * 4);
        f(reinterpret_cast<void**>(&c->ub_ngroups), 16);
        // the whole-grid path for large groups: per-CTA partial sums and digit counts, barrier
        f(reinterpret_cast<void**>(&c->ub_part), size_t(kUnbindGridCtaCap) * 16 * 8);
        f(reinterpret_cast<void**>(&c->ub_hist), size_t(kUnbindGridCtaCap) * 2 * 256 * 4);
        f(reinterpret_cast<void**>(&c->ub_bar), 16);
    }
    f(reinterpret_cast<void**>(&c->scan_tmp), z.scan_words * 4);
    f(reinterpret_cast<void**>(&c->grid), size_t(z.cells) * 8);
    f(reinterpret_cast<void**>(&c->cwt), size_t(z.cells) * 4);
    f(reinterpret_cast<void**>(&c->label), size_t(z.cells) * 4);
    f(reinterpret_cast<void**>(&c->table_dev), table_slot_floats(max_ng) * kTableSlots * 4);
}

void release(cwthf_ctx* c) {
    for_each_buffer(c, c->max_ng, c->max_np, c->max_scales, c->flags, [](void** p, size_t) {
        if (*p) cudaFree(*p);
        *p = nullptr;
    });
    if (c->h_status) cudaFreeHost(c->h_status);
    c->h_status = nullptr;
    if (c->table_host) cudaFreeHost(c->table_host);
    c->table_host = nullptr;
    free_tables(c);
}

int check_common(const cwthf_ctx* ctx, int ng, double L) {
    if (!ctx) return CWTHF_E_INVALID_ARG;
    if (!(L > 0) || !std::isfinite(L)) return CWTHF_E_INVALID_ARG;
    int rc = check_ng(ng);
    if (rc) return rc;
    if (ng > ctx->max_ng) return CWTHF_E_UNSUPPORTED_SIZE;
    return CWTHF_OK;
}

int check_particles(const cwthf_ctx* ctx, const float* pos, int64_t np, double mass_unit) {
    if (np < 0 || np > ctx->max_np) return CWTHF_E_INVALID_ARG;
    if (np > 0 && !pos) return CWTHF_E_INVALID_ARG;
    if (!(mass_unit > 0) || !std::isfinite(mass_unit)) return CWTHF_E_INVALID_ARG;
    return CWTHF_OK;
}

cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

}  // namespace
}  // namespace cwthf

using namespace cwthf;

extern "C" {

void cwthf_default_params(double w, cwthf_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->w = w;
    p->cwt_min = 0.0f;
    p->dens_th = 4.0;
    p->particle_th = 15;
}

int cwthf_check_ng(int ng) { return check_ng(ng) ? CWTHF_E_UNSUPPORTED_SIZE : CWTHF_OK; }

int cwthf_workspace_bytes_ex(int max_ng, int64_t max_np, int max_scales, unsigned flags, size_t* out) {
    if (!out || max_np < 0 || max_np >= (int64_t(1) << 31) || max_scales < 1 || (flags & ~kCreateFlags))
        return CWTHF_E_INVALID_ARG;
    if (check_ng(max_ng)) return CWTHF_E_UNSUPPORTED_SIZE;
    cwthf_ctx probe;
    size_t total = 0;
    for_each_buffer(&probe, max_ng, max_np, max_scales, flags,
                    [&](void**, size_t b) { total += (b + 255) / 256 * 256; });
    *out = total;
    return CWTHF_OK;
}

int cwthf_workspace_bytes(int max_ng, int64_t max_np, int max_scales, size_t* out) {
    return cwthf_workspace_bytes_ex(max_ng, max_np, max_scales, 0u, out);
}

int cwthf_create(int device, int max_ng, int64_t max_np, int max_scales, cwthf_ctx** out) {
    return cwthf_create_ex(device, max_ng, max_np, max_scales, 0u, out);
}

int cwthf_create_ex(int device, int max_ng, int64_t max_np, int max_scales, unsigned flags, cwthf_ctx** out) {
    if (!out) return CWTHF_E_INVALID_ARG;
    *out = nullptr;
    if (max_np < 0 || max_np >= (int64_t(1) << 31) || max_scales < 1 || (flags & ~kCreateFlags))
        return CWTHF_E_INVALID_ARG;
    if (check_ng(max_ng)) return CWTHF_E_UNSUPPORTED_SIZE;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return CWTHF_E_CUDA;
    DeviceGuard g(device);
    if (!g.ok) return CWTHF_E_CUDA;
    cwthf_ctx* c = new (std::nothrow) cwthf_ctx;
    if (!c) return CWTHF_E_OOM;
    c->device = device;
    c->max_ng = max_ng;
    c->max_np = max_np;
    c->max_scales = max_scales;
    c->flags = flags;
    if (cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        (c->fallback_blocks = fallback_blocks(c->sm_count)) <= 0 ||
        ((flags & CWTHF_CREATE_UNBIND) &&
         (c->ub_grid_blocks = std::min(unbind_grid_blocks(c->sm_count), kUnbindGridCtaCap)) <= 0)) {
        delete c;
        return CWTHF_E_CUDA;
    }
    bool failed = false;
    for_each_buffer(c, max_ng, max_np, max_scales, flags, [&](void** p, size_t b) {
        if (failed) return;
        if (cudaMalloc(p, b) != cudaSuccess) {
            *p = nullptr;
            failed = true;
        }
    });
    if (!failed && cudaMallocHost(&c->h_status, sizeof(int) * 2) != cudaSuccess) failed = true;
    c->table_slot_floats = table_slot_floats(max_ng);
    if (!failed && cudaMallocHost(&c->table_host, c->table_slot_floats * kTableSlots * 4) != cudaSuccess) failed = true;
    if (!failed && init_tables(c) != CWTHF_OK) failed = true;
    if (!failed) {
        Sizes z = sizes_for(max_ng, max_np);
        c->scan_tmp_cap = z.scan_words;
        if (cudaMemset(c->d_status, 0, sizeof(int) * 4) != cudaSuccess) failed = true;
    }
    if (failed) {
        cudaGetLastError();  // clear the sticky allocation error
        release(c);
        delete c;
        return CWTHF_E_OOM;
    }
    *out = c;
    return CWTHF_OK;
}

void cwthf_destroy(cwthf_ctx* ctx) {
    if (!ctx) return;
    DeviceGuard g(ctx->device);
    cudaDeviceSynchronize();
    cwthf_profile(ctx, 0);
    for (cudaEvent_t e : ctx->prof_pool) cudaEventDestroy(e);
    ctx->prof_pool.clear();
    release(ctx);
    delete ctx;
}

int cwthf_deposit(cwthf_ctx* ctx, const float* pos, const float* mass, double mass_unit, int64_t np, double L,
                  int ng, int64_t* grid, int64_t* mtot, void* stream) {
    int rc = check_common(ctx, ng, L);
    if (!rc) rc = check_particles(ctx, pos, np, mass_unit);
    if (!rc && !grid) rc = CWTHF_E_INVALID_ARG;
    if (rc) return rc;
    DeviceGuard g(ctx->device);
    Range r("cwthf_deposit (S1)");
    return deposit_impl(ctx, pos, mass, mass_unit, np, L, ng, grid, mtot, as_stream(stream));
}

int cwthf_transform(cwthf_ctx* ctx, const int64_t* grid, int ng, double L, double mass_unit, double w, float* cwt,
                    void* stream) {
    int rc = check_common(ctx, ng, L);
    if (rc) return rc;
    if (!grid || !cwt || !(w > 0) || !std::isfinite(w) || !(mass_unit > 0)) return CWTHF_E_INVALID_ARG;
    DeviceGuard g(ctx->device);
    cudaStream_t s = as_stream(stream);
    const float* wtab = nullptr;
    Range r("cwthf_transform (S2-S4)");
    rc = transform_tables(ctx, ng, L, &w, 1, &wtab, s);
    if (!rc) rc = transform_forward_xy(ctx, grid, ng, ctx->spec, s);
    if (!rc) rc = transform_wavelet_inverse(ctx, ctx->spec, ctx->spec, ng, L, w, mass_unit, wtab, cwt, s);
    return rc;
}

int cwthf_transform_stencil(cwthf_ctx* ctx, const int64_t* grid, int ng, double L, double mass_unit, double w, int R,
                            float* cwt, void* stream) {
    int rc = check_common(ctx, ng, L);
    if (rc) return rc;
    if (!grid || !cwt || !(w > 0) || !std::isfinite(w) || !(mass_unit > 0) || !std::isfinite(mass_unit) || R < 0 ||
        R > CWTHF_MAX_STENCIL_R || 2 * R + 1 > ng)
        return CWTHF_E_INVALID_ARG;
    DeviceGuard g(ctx->device);
    Range r("cwthf_transform_stencil (S2-S4, direct space)");
    return transform_stencil_impl(ctx, grid, ng, L, mass_unit, w, R, cwt, as_stream(stream));
}

int cwthf_prepare(cwthf_ctx* ctx, int ng, double L, const double* w, int n_scales, void* stream) {
    int rc = check_common(ctx, ng, L);
    if (rc) return rc;
    if (n_scales < 0 || (n_scales > 0 && !w)) return CWTHF_E_INVALID_ARG;
    for (int i = 0; i < n_scales; i++)
        if (!(w[i] > 0) || !std::isfinite(w[i])) return CWTHF_E_INVALID_ARG;
    DeviceGuard g(ctx->device);
    std::vector<const float*> wtab(size_t(std::max(n_scales, 1)));
    return transform_tables(ctx, ng, L, w, n_scales, wtab.data(), as_stream(stream));
}

int cwthf_segment(cwthf_ctx* ctx, const float* cwt, int ng, float cwt_min, int32_t* cell_label, void* stream) {
    int rc = check_common(ctx, ng, 1.0);
    if (rc) return rc;
    if (!cwt || !cell_label || std::isnan(cwt_min)) return CWTHF_E_INVALID_ARG;
    DeviceGuard g(ctx->device);
    Range r("cwthf_segment (S5-S6)");
    return segment_impl(ctx, cwt, ng, cwt_min, cell_label, false, as_stream(stream));
}

int cwthf_unbind(cwthf_ctx* ctx, const float* pos, const float* vel, const float* mass, double mass_unit, int64_t np,
                 double L, double G, const int32_t* group, int64_t n_groups, int max_iter, int32_t* group_out,
                 int64_t* n_kept, int32_t* iters, void* stream) {
    if (!ctx || !(ctx->flags & CWTHF_CREATE_UNBIND)) return CWTHF_E_INVALID_ARG;
    int rc = check_particles(ctx, pos, np, mass_unit);
    if (rc) return rc;
    if ((np > 0 && (!vel || !group || !group_out)) || n_groups < 0 || (n_groups > 0 && (!n_kept || !iters)) ||
        max_iter < 1 || !(L > 0) || !std::isfinite(L) || !(G >= 0) || !std::isfinite(G))
        return CWTHF_E_INVALID_ARG;
    if (n_groups > int64_t(ctx->max_ng) * ctx->max_ng * ctx->max_ng / 8 + 8) return CWTHF_E_CAPACITY;
    DeviceGuard g(ctx->device);
    Range r("cwthf_unbind (Sec. 2.3)");
    return unbind_impl(ctx, pos, vel, mass, mass_unit, np, L, G, group, n_groups, max_iter, group_out, n_kept, iters,
                       as_stream(stream));
}

int cwthf_segment_sizes(cwthf_ctx* ctx, int32_t* seeds, int64_t* n_cells, int64_t cap, int64_t* n_seeds,
                        void* stream) {
    if (!ctx || cap < 0 || (cap > 0 && (!seeds || !n_cells)) || !n_seeds) return CWTHF_E_INVALID_ARG;
    DeviceGuard g(ctx->device);
    return segment_sizes_impl(ctx, seeds, n_cells, cap, n_seeds, as_stream(stream));
}

int cwthf_assign(cwthf_ctx* ctx, const float* pos, const float* mass, double mass_unit, int64_t np, double L, int ng,
                 const int32_t* cell_label, const float* cwt, const cwthf_params* params, int32_t* halo_id,
                 cwthf_halo* cat, int64_t cat_cap, int64_t* n_halo, void* stream) {
    int rc = check_common(ctx, ng, L);
    if (!rc) rc = check_particles(ctx, pos, np, mass_unit);
    if (rc) return rc;
    if (!cell_label || !params || (np > 0 && !halo_id) || cat_cap < 0 || (cat_cap > 0 && !cat) || !n_halo ||
        std::isnan(params->dens_th))
        return CWTHF_E_INVALID_ARG;
    DeviceGuard g(ctx->device);
    Range r("cwthf_assign (S7-S8)");
    return assign_impl(ctx, pos, mass, mass_unit, np, L, ng, cell_label, cwt, params, 0, 1, halo_id, cat, cat_cap,
                       n_halo, false, false, as_stream(stream));
}

int cwthf_find(cwthf_ctx* ctx, const float* pos, const float* mass, double mass_unit, int64_t np, double L, int ng,
               const cwthf_params* params, int n_scales, int32_t* halo_id, cwthf_halo* cat, int64_t cat_cap,
               int64_t* n_halo, void* stream) {
    int rc = check_common(ctx, ng, L);
    if (!rc) rc = check_particles(ctx, pos, np, mass_unit);
    if (rc) return rc;
    if (!params || n_scales < 1 || n_scales > ctx->max_scales || (np > 0 && !halo_id) || cat_cap < 0 ||
        (cat_cap > 0 && !cat) || !n_halo)
        return CWTHF_E_INVALID_ARG;
    for (int i = 0; i < n_scales; i++)
        if (!(params[i].w > 0) || !std::isfinite(params[i].w) || std::isnan(params[i].cwt_min) ||
            std::isnan(params[i].dens_th))
            return CWTHF_E_INVALID_ARG;
    DeviceGuard g(ctx->device);
    cudaStream_t s = as_stream(stream);
    std::vector<double> ws(n_scales);
    std::vector<const float*> wtab(n_scales);
    for (int i = 0; i < n_scales; i++) ws[i] = params[i].w;
    Range r("cwthf_find");
    rc = transform_tables(ctx, ng, L, ws.data(), n_scales, wtab.data(), s);
    if (!rc) {
        Range r1("S1 deposit");
        rc = deposit_impl(ctx, pos, mass, mass_unit, np, L, ng, ctx->grid, nullptr, s);
    }
    if (!rc) {
        Range r2("S2 forward FFT (x, y)");
        rc = transform_forward_xy(ctx, ctx->grid, ng, ctx->spec, s);
    }
    for (int i = 0; i < n_scales && !rc; i++) {
        float2* dst = n_scales > 1 ? ctx->spec2 : ctx->spec;
        {
            Range r3("S2-S4 z FFT, wavelet multiply, inverse FFT");
            rc = transform_wavelet_inverse(ctx, ctx->spec, dst, ng, L, params[i].w, mass_unit, wtab[i], ctx->cwt, s);
        }
        if (!rc) {
            Range r5("S5-S6 maxima and segmentation");
            rc = segment_impl(ctx, ctx->cwt, ng, params[i].cwt_min, ctx->label, true, s);
        }
        if (!rc) {
            Range r7("S7-S8 assignment and halo sums");
            rc = assign_impl(ctx, pos, mass, mass_unit, np, L, ng, ctx->label, ctx->cwt, &params[i], i, n_scales,
                             halo_id, cat + int64_t(i) * cat_cap, cat_cap, n_halo + i, true, true, s);
        }
    }
    return rc;
}

int cwthf_find_multiscale(cwthf_ctx* ctx, const float* pos, const float* mass, double mass_unit, int64_t np, double L,
                          int n_scales, const double* w, const int* ng, float cwt_min, double dens_th,
                          int64_t particle_th, const float* vel, double G, int max_iter, int32_t* halo_id,
                          cwthf_ms_halo* cat, int64_t cat_cap, int64_t* n_halo, void* stream) {
    if (!ctx || !w || !ng || n_scales < 1 || ctx->max_scales < 2) return CWTHF_E_INVALID_ARG;
    if (vel && (!(ctx->flags & CWTHF_CREATE_UNBIND) || max_iter < 1 || !(G >= 0) || !std::isfinite(G)))
        return CWTHF_E_INVALID_ARG;
    int rc = check_particles(ctx, pos, np, mass_unit);
    if (rc) return rc;
    if ((np > 0 && !halo_id) || cat_cap < 0 || (cat_cap > 0 && !cat) || !n_halo || std::isnan(cwt_min) ||
        std::isnan(dens_th))
        return CWTHF_E_INVALID_ARG;
    for (int j = 0; j < n_scales; j++) {
        if ((rc = check_common(ctx, ng[j], L))) return rc;
        if (!(w[j] > 0) || !std::isfinite(w[j])) return CWTHF_E_INVALID_ARG;
    }
    DeviceGuard g(ctx->device);
    cudaStream_t s = as_stream(stream);
    Range r("cwthf_find_multiscale");
    // every scale's tables before anything is queued
    for (int j = 0; j < n_scales && !rc; j++) {
        const float* wt = nullptr;
        rc = transform_tables(ctx, ng[j], L, &w[j], 1, &wt, s);
    }
    if (rc) return rc;
    // the two fields kept at a time: the CWT buffer and the second spectrum
    float* field[2] = {ctx->cwt, reinterpret_cast<float*>(ctx->spec2)};
    int32_t* pslot = ctx->part_slot + std::max<int64_t>(np, 1);
    unsigned long long* mtot_all = ctx->d_mtot + 1;  // total mass of all particles
    cudaError_t e = cudaMemsetAsync(n_halo, 0, sizeof(int64_t), s);
    if (e == cudaSuccess && np > 0) e = cudaMemsetAsync(halo_id, 0xff, size_t(np) * sizeof(int32_t), s);
    if (e != cudaSuccess) return cuda_status(e);
    for (int j = 0; j <= n_scales && !rc; j++) {
        if (j < n_scales) {  // deposit and CWT of scale j
            Range r1("scale: deposit and CWT");
            const float* wt = nullptr;
            rc = transform_tables(ctx, ng[j], L, &w[j], 1, &wt, s);
            if (!rc) rc = deposit_impl(ctx, pos, mass, mass_unit, np, L, ng[j], ctx->grid, nullptr, s);
            if (!rc && j == 0 &&
                (e = cudaMemcpyAsync(mtot_all, ctx->d_mtot, sizeof(unsigned long long), cudaMemcpyDeviceToDevice,
                                     s)) != cudaSuccess)
                rc = cuda_status(e);
            if (!rc) rc = transform_forward_xy(ctx, ctx->grid, ng[j], ctx->spec, s);
            if (!rc) rc = transform_wavelet_inverse(ctx, ctx->spec, ctx->spec, ng[j], L, w[j], mass_unit, wt, field[j & 1], s);
        }
        if (j >= 1 && !rc) {  // decide scale j - 1 against scale j's field
            Range r2("scale: cross-scale check, thresholds, halo ids");
            const bool last = j == n_scales;
            rc = ms_finalize(ctx, pos, mass, np > 0 ? vel : nullptr, G, max_iter, np, L, ng[j - 1], mass_unit,
                             field[(j - 1) & 1], last ? nullptr : field[j & 1],
                             last ? 0 : ng[j], j - 1, dens_th, particle_th, pslot, mtot_all, halo_id, cat, cat_cap,
                             n_halo, s);
        }
        if (j < n_scales && !rc) {  // segments and groups of scale j
            Range r3("scale: segmentation and group sums");
            rc = segment_impl(ctx, field[j & 1], ng[j], cwt_min, ctx->label, true, s);
            if (!rc) rc = ms_scale_sums(ctx, pos, mass, mass_unit, np, L, ng[j], halo_id, pslot, s);
        }
    }
    return rc;
}

int cwthf_sync(cwthf_ctx* ctx, void* stream) {
    if (!ctx) return CWTHF_E_INVALID_ARG;
    DeviceGuard g(ctx->device);
    cudaStream_t s = as_stream(stream);
    if (cudaStreamSynchronize(s) != cudaSuccess) return CWTHF_E_CUDA;
    if (cudaMemcpyAsync(ctx->h_status, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemsetAsync(ctx->d_status, 0, sizeof(int), s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
        return CWTHF_E_CUDA;
    return *ctx->h_status;
}

const char* cwthf_error_string(int code) {
    switch (code) {
        case CWTHF_OK: return "ok";
        case CWTHF_E_INVALID_ARG: return "invalid argument";
        case CWTHF_E_UNSUPPORTED_SIZE: return "unsupported grid size (need an even ng, 8 <= ng <= 1152, within the context's limits)";
        case CWTHF_E_OVERFLOW: return "integer mass budget exceeded (m_q >= 2^31 or sum m_q >= 2^33)";
        case CWTHF_E_OOM: return "device allocation failed";
        case CWTHF_E_CUDA: return "CUDA runtime error";
        case CWTHF_E_NOT_CONVERGED: return "label propagation did not converge within its round limit";
        case CWTHF_E_TIMEOUT: return "a bounded device wait timed out";
        case CWTHF_E_CAPACITY: return "more halos than the catalogue capacity";
        case CWTHF_E_BAD_INPUT: return "non-finite or out-of-range input value";
        case CWTHF_E_SCRATCH_LIMIT: return "size beyond the fixed scratch of cwthf_deposit_noalloc (ng <= 128, np <= 262144)";
        case CWTHF_E_TABLE_CACHE: return "no free FFT / wavelet table slot (all in use by captured graphs, or a capture needs a new one)";
        case CWTHF_E_INDEX: return "an index out of range was caught by the checked build (results unspecified)";
        default: return "unknown status";
    }
}

int64_t cwthf_launch_count(const cwthf_ctx* ctx) { return ctx ? ctx->launches.load() : 0; }

int cwthf_set_fft_plan(cwthf_ctx* ctx, int ng, int which, int C, const int* radices, int n_radices) {
    if (!ctx || n_radices < 0 || n_radices > 3) return CWTHF_E_INVALID_ARG;
    int rc = check_common(ctx, ng, 1.0);
    if (rc) return rc;
    return set_fft_plan(ctx, ng, which, C, radices, n_radices);
}

int cwthf_debug_set(cwthf_ctx* ctx, int key, int64_t value) {
    if (!ctx) return CWTHF_E_INVALID_ARG;
    switch (key) {
        case CWTHF_DEBUG_JUMP_ROUNDS:
            if (value < 0 || value > kMaxJumpRounds) return CWTHF_E_INVALID_ARG;
            ctx->dbg_jump_rounds = int(value);
            return CWTHF_OK;
        case CWTHF_DEBUG_CHASE_LIMIT:
            if (value < 1 || value > kDefaultChaseLimit) return CWTHF_E_INVALID_ARG;
            ctx->dbg_chase_limit = int(value);
            return CWTHF_OK;
        case CWTHF_DEBUG_TMA_NO_COPY:
            ctx->dbg_tma_no_copy = value != 0;
            return CWTHF_OK;
        case CWTHF_DEBUG_UNBIND_GRID_MIN:
            if (value < 1 || value >= (int64_t(1) << 31)) return CWTHF_E_INVALID_ARG;
            ctx->dbg_unbind_grid_min = value;
            return CWTHF_OK;
        default:
            return CWTHF_E_INVALID_ARG;
    }
}

int cwthf_debug_get(cwthf_ctx* ctx, int key, int64_t* value, void* stream) {
    if (!ctx || !value) return CWTHF_E_INVALID_ARG;
    switch (key) {
        case CWTHF_DEBUG_JUMP_ROUNDS: *value = ctx->dbg_jump_rounds; return CWTHF_OK;
        case CWTHF_DEBUG_CHASE_LIMIT: *value = ctx->dbg_chase_limit; return CWTHF_OK;
        case CWTHF_DEBUG_TMA_NO_COPY: *value = ctx->dbg_tma_no_copy; return CWTHF_OK;
        case CWTHF_DEBUG_UNBIND_GRID_MIN: *value = ctx->dbg_unbind_grid_min; return CWTHF_OK;
        case CWTHF_DEBUG_CHECKED: *value = kCheckedBuild ? 1 : 0; return CWTHF_OK;
        case CWTHF_DEBUG_TABLE_FILLS: {
            std::lock_guard<std::mutex> lk(ctx->table_mu);
            *value = int64_t(ctx->table_fills);
            return CWTHF_OK;
        }
        case CWTHF_DEBUG_FALLBACK_RAN: {
            DeviceGuard g(ctx->device);
            cudaStream_t s = as_stream(stream);
            int v = 0;
            if (cudaMemcpyAsync(ctx->h_status + 1, ctx->jump_changed, sizeof(int), cudaMemcpyDeviceToHost, s) !=
                    cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess)
                return CWTHF_E_CUDA;
            v = ctx->h_status[1];
            *value = v != 0;
            return CWTHF_OK;
        }
        default:
            return CWTHF_E_INVALID_ARG;
    }
}

int cwthf_profile(cwthf_ctx* ctx, int enable) {
    if (!ctx) return CWTHF_E_INVALID_ARG;
    DeviceGuard g(ctx->device);
    for (auto& r : ctx->prof_pending) {
        cudaEventSynchronize(r.b);
        ctx->prof_pool.push_back(r.a);
        ctx->prof_pool.push_back(r.b);
    }
    ctx->prof_pending.clear();
    ctx->prof_names.clear();
    ctx->prof_ms.clear();
    ctx->prof_n.clear();
    ctx->prof_on = enable != 0;
    return CWTHF_OK;
}

int cwthf_profile_count(cwthf_ctx* ctx) {
    if (!ctx) return -CWTHF_E_INVALID_ARG;
    DeviceGuard g(ctx->device);
    int rc = CWTHF_OK;
    for (auto& r : ctx->prof_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess)
            rc = CWTHF_E_CUDA;
        size_t k = 0;
        while (k < ctx->prof_names.size() && std::strcmp(ctx->prof_names[k], r.name) != 0) k++;
        if (k == ctx->prof_names.size()) {
            ctx->prof_names.push_back(r.name);
            ctx->prof_ms.push_back(0.0);
            ctx->prof_n.push_back(0);
        }
        ctx->prof_ms[k] += ms;
        ctx->prof_n[k] += 1;
        ctx->prof_pool.push_back(r.a);
        ctx->prof_pool.push_back(r.b);
    }
    ctx->prof_pending.clear();
    return rc ? -rc : int(ctx->prof_names.size());
}

int cwthf_profile_read(const cwthf_ctx* ctx, int i, const char** name, double* total_ms, int64_t* launches) {
    if (!ctx || i < 0 || size_t(i) >= ctx->prof_names.size()) return CWTHF_E_INVALID_ARG;
    if (name) *name = ctx->prof_names[i];
    if (total_ms) *total_ms = ctx->prof_ms[i];
    if (launches) *launches = ctx->prof_n[i];
    return CWTHF_OK;
}

}  // extern "C"
