// internal.cuh -- declarations shared by the CUDA translation units of
// libcwthf.so (not part of the public ABI; see include/cwthf.h).
#pragma once

#include <cuda/atomic>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "../../include/cwthf.h"

namespace cwthf {

constexpr int kFracBits = CWTHF_FRAC_BITS;
constexpr int64_t kFracOne = int64_t(1) << kFracBits;

// Deposit tiles: the grid is cut into tiles of kDepTX x kDepTY x kDepTZ cells
// (the last tile along an axis may be partial).
constexpr int kDepTX = 32, kDepTY = 8, kDepTZ = 8;
constexpr int kDepClasses = 8;  // boundary class bits (x, y, z) per particle
// Records of a deposit tile per CTA pass: denser tiles are split into parts.
// The records reaching into all tiles number at most 8 np (a particle reaches
// its own tile and at most 7 neighbours), so the parts after each tile's
// first number at most 8 np / kTileSplit.
constexpr uint32_t kTileSplit = 4096;
inline int64_t tile_parts_cap(int64_t np) { return 8 * (np > 0 ? np : 1) / kTileSplit + 1; }

// A binned particle record: its three fixed-point coordinates q (each below
// ng * 2^10 <= 2^20) in 21-bit fields, x lowest.
constexpr int kRecBits = 21;
static_assert(int64_t(CWTHF_MAX_NG) * (int64_t(1) << CWTHF_FRAC_BITS) <= (int64_t(1) << kRecBits),
              "record fields too narrow for the largest grid");
__host__ __device__ __forceinline__ unsigned long long pack_rec(int64_t qx, int64_t qy, int64_t qz) {
    return (unsigned long long)qx | ((unsigned long long)qy << kRecBits) | ((unsigned long long)qz << (2 * kRecBits));
}
__host__ __device__ __forceinline__ int rec_q(unsigned long long e, int d) {
    return int((e >> (kRecBits * d)) & ((1ull << kRecBits) - 1));
}

// Pointer-doubling rounds of the segmentation's fallback: round r moves every
// unfinished pointer 2^(r-1) or more links further, so 31 rounds end any chain
// of a grid of at most 2^30 cells.
constexpr int kMaxJumpRounds = 31;
// The segmentation's control words (ctx->jump_changed, cleared per call):
// [0 .. kMaxJumpRounds] "a pointer is still flagged" after the resolve pass
// (0) and after each doubling round, then the resolve pass's tile counter and
// the fallback's grid-barrier state (arrivals, generation).
constexpr int kJumpTileCounter = kMaxJumpRounds + 1;
constexpr int kJumpBarrier = kMaxJumpRounds + 2;
constexpr int kJumpWords = kMaxJumpRounds + 4;
// Default length of the resolve pass's bounded chain walks.
constexpr int kDefaultChaseLimit = 64;

// Groups of the self-boundness check with more members than this are
// processed by the whole grid, one at a time; smaller ones by one CTA each.
constexpr int64_t kUnbindGridMin = 1 << 16;
// Most CTAs of that whole-grid launch (its per-CTA scratch is sized for them).
constexpr int kUnbindGridCtaCap = 1024;

// A bounded device wait gives up after this many polls.
constexpr long long kSpinLimit = 1ll << 20;

struct Tables;  // FFT twiddles of one grid size (fft.cu)

// Table slots of a context, allocated by cwthf_create: FFT twiddles (per grid
// size) and wavelet spectra (per grid size, box and scale), each slot holding
// up to 3 * max_ng floats on the device, with a pinned host staging copy.
constexpr int kTableSlots = 48;
constexpr int kTableTwiddles = 0, kTableWavelet = 1;
struct TableSlot {
    int kind = -1;  // -1: free
    int ng = 0;
    double L = 0.0, w = 0.0;
    unsigned long long last_use = 0;
    bool graph_ref = false;          // read by work captured into a CUDA graph: never reused
    bool on_device = false;          // a copy was queued outside any capture
    cudaEvent_t filled = nullptr;    // recorded after that copy
};

struct cwthf_ctx_impl;

// Shape of one complex half-spectrum workspace [ng][ng][pitch] (float2).
inline int spec_pitch(int ng) {
    int m = ng / 2 + 1;
    return (m % 2) ? m + 1 : m;  // even number of complex -> 16-byte aligned rows
}
inline size_t spec_bytes(int ng) { return size_t(ng) * ng * spec_pitch(ng) * 8; }

inline int div_up(int64_t a, int64_t b) { return int((a + b - 1) / b); }

struct DepositGeom {
    int ng, ntx, nty, ntz;
    int64_t ntiles;
};
inline DepositGeom deposit_geom(int ng) {
    DepositGeom g;
    g.ng = ng;
    g.ntx = div_up(ng, kDepTX);
    g.nty = div_up(ng, kDepTY);
    g.ntz = div_up(ng, kDepTZ);
    g.ntiles = int64_t(g.ntx) * g.nty * g.ntz;
    return g;
}

// Per-slot accumulators of the halo reduction (one slot per seed).
struct HaloAcc {
    unsigned long long n_part;
    unsigned long long mq;
    long long mom[3];
    unsigned long long n_cells;
};

}  // namespace cwthf

// The opaque context of the public ABI.
struct cwthf_ctx {
    int device = 0;
    int max_ng = 0;
    int64_t max_np = 0;
    int max_scales = 1;
    unsigned flags = 0;  // CWTHF_CREATE_* given to cwthf_create_ex
    int sm_count = 0;

    int* d_status = nullptr;   // first device-side error since the last cwthf_sync
    int* h_status = nullptr;   // pinned mirror

    // deposit scratch
    uint32_t* dep_count = nullptr;   // [max_tiles * 8 + 1]
    uint32_t* dep_off = nullptr;     // [max_tiles * 8 + 1]
    uint32_t* dep_cursor = nullptr;  // [max_tiles * 8]
    unsigned long long* dep_rec = nullptr;  // [max_np] packed fixed-point records (pack_rec)
    uint32_t* dep_mq = nullptr;             // [max_np] integer masses of the records
    uint32_t* part_rec = nullptr;           // [max_np] record position of each particle (~0u: not binned)
    unsigned long long* d_mtot = nullptr;   // [1] sum of m_q of the last deposit / assign

    // transform scratch
    float2* spec = nullptr;    // complex half spectrum [ng][ng][pitch]
    float2* spec2 = nullptr;   // second spectrum (multi-scale), or nullptr

    // segmentation / assignment scratch
    uint32_t* seed_bits = nullptr;    // [ng^3 / 32 + 1] seed bitmap
    uint32_t* seed_prefix = nullptr;  // [ng^3 / 32 + 1] exclusive popcount prefix
    uint32_t* seed_cells = nullptr;   // [ng^3] a seed's segment cell count at the seed's cell (valid at seeds only)
    int32_t* seed_list = nullptr;     // [ng^3 / 8 + 1] seed cell of each slot
    uint32_t* n_seeds = nullptr;      // [1]
    cwthf::HaloAcc* acc = nullptr;    // [ng^3 / 8 + 1]
    uint32_t* keep_off = nullptr;     // [ng^3 / 8 + 2] kept-halo prefix
    int32_t* slot_halo = nullptr;     // [max_scales][ng^3 / 8 + 8] seed of each kept slot, -1 otherwise
    int32_t* part_slot = nullptr;     // [max_scales][max_np] record slots (-1: none), then [max_np][1|2|4k] halo ids
    int* jump_changed = nullptr;      // [kJumpWords] segmentation control words
    uint32_t* scan_tmp = nullptr;     // block sums of the device scan
    size_t scan_tmp_cap = 0;          // words

    // self-boundness check scratch (cwthf_unbind)
    uint32_t* ub_off = nullptr;   // [max groups + 2] members per group, then their offsets
    uint32_t* ub_cur = nullptr;   // [max groups + 1] scatter cursors
    int32_t* ub_mem = nullptr;    // [max_np] members, grouped
    uint64_t* ub_key = nullptr;   // [2 max_np] sort keys
    int32_t* ub_val = nullptr;    // [2 max_np] sort values
    int32_t* ub_grp = nullptr;    // [max_np] the multi-scale loop's groups per particle
    int32_t* ub_out = nullptr;    // [max_np] their groups after the check
    int64_t* ub_nk = nullptr;     // [max groups] members kept per group
    int32_t* ub_it = nullptr;     // [max groups] rounds per group
    uint32_t* ub_keep = nullptr;  // [max groups + 2] groups that stay, then their ranks
    uint32_t* ub_ngroups = nullptr;  // [1] groups of the check (device count)
    unsigned long long* dep_parts = nullptr;  // [tile_parts_cap(max_np)] (tile, part) of dense deposit tiles
    uint32_t* dep_nparts = nullptr;          // [1] parts listed
    double* ub_part = nullptr;       // [ub_grid_blocks][16] per-CTA partial sums of the whole-grid path
    uint32_t* ub_hist = nullptr;     // [2][ub_grid_blocks][256] per-CTA digit counts of its radix sort
    unsigned* ub_bar = nullptr;      // [2] its grid barrier
    int ub_grid_blocks = 0;          // CTAs of the whole-grid path's cooperative launch

    // cwthf_find internals
    int64_t* grid = nullptr;
    float* cwt = nullptr;
    int32_t* label = nullptr;

    int fallback_blocks = 0;          // CTAs of the cooperative segmentation fallback

    // test and fault-injection settings (cwthf_debug_set)
    int dbg_jump_rounds = cwthf::kMaxJumpRounds;
    int dbg_chase_limit = cwthf::kDefaultChaseLimit;
    int dbg_tma_no_copy = 0;  // one-shot: the next y/z FFT pass runs one CTA without its copy
    int64_t dbg_unbind_grid_min = cwthf::kUnbindGridMin;  // groups above this size take the whole grid

    std::atomic<int64_t> launches{0};

    // optional per-kernel CUDA-event timing (cwthf_profile)
    struct ProfRec {
        const char* name;
        cudaEvent_t a, b;
    };
    bool prof_on = false;
    std::vector<ProfRec> prof_pending;
    std::vector<cudaEvent_t> prof_pool;
    std::vector<const char*> prof_names;
    std::vector<double> prof_ms;
    std::vector<int64_t> prof_n;

    // FFT plans chosen by the caller (cwthf_set_fft_plan) instead of the
    // built-in rule, per (grid size, pass): C, number of stages, radices
    struct PlanOverride {
        int ng, which, C, nst, rad[3];
    };
    std::vector<PlanOverride> fft_plans;

    std::mutex table_mu;
    float* table_dev = nullptr;   // [kTableSlots][table_slot_floats]
    float* table_host = nullptr;  // pinned staging, same shape
    size_t table_slot_floats = 0;
    unsigned long long table_clock = 0;
    unsigned long long table_fills = 0;  // slots filled since creation
    cwthf::TableSlot table_slot[cwthf::kTableSlots];
};

namespace cwthf {

// ---- status helpers ---------------------------------------------------------
__device__ __forceinline__ void set_status(int* st, int code) { atomicCAS(st, 0, code); }

// Checked builds (CWTHF_CHECKED): a data-driven index -- one read from device
// memory rather than formed from loop bounds -- is tested before use; one out
// of [0, n) records CWTHF_E_INDEX and the access is skipped.  Elsewhere the
// test compiles away.
#ifdef CWTHF_CHECKED
constexpr bool kCheckedBuild = true;
#else
constexpr bool kCheckedBuild = false;
#endif
__device__ __forceinline__ bool index_ok(long long i, long long n, int* status) {
    if (!kCheckedBuild || (i >= 0 && i < n)) return true;
    set_status(status, CWTHF_E_INDEX);
    return false;
}

// Bounded grid-wide barrier for kernels launched cooperatively (every CTA
// resident).  bar[0] counts arrivals, bar[1] is the generation.  The wait
// gives up after kSpinLimit polls, records CWTHF_E_TIMEOUT and returns false;
// the CTA then leaves the kernel.  Data that other CTAs wrote before the
// barrier is read with L1-bypassing loads (__ldcg) after it.
__device__ __forceinline__ bool grid_sync(unsigned* bar, int* status) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        cuda::atomic_ref<unsigned, cuda::thread_scope_device> cnt(bar[0]), gen(bar[1]);
        const unsigned g = gen.load(cuda::memory_order_acquire);
        __threadfence();
        if (cnt.fetch_add(1u, cuda::memory_order_acq_rel) == gridDim.x - 1) {
            cnt.store(0u, cuda::memory_order_relaxed);
            gen.store(g + 1u, cuda::memory_order_release);
        } else {
            long long it = 0;
            while (gen.load(cuda::memory_order_acquire) == g) {
                if (++it > kSpinLimit) {
                    ok = 0;
                    set_status(status, CWTHF_E_TIMEOUT);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

// Slot (rank among all seeds, in cell order) of seed cell `lab`, from the seed
// bitmap and its per-word popcount prefix; false if lab is not a seed or its
// slot is beyond the number of slots in use.
__device__ __forceinline__ bool seed_slot(const uint32_t* bits, const uint32_t* prefix, const uint32_t* n_slots,
                                          int32_t lab, uint32_t& slot) {
    uint32_t w = bits[lab >> 5];
    uint32_t m = 1u << (lab & 31);
    slot = prefix[lab >> 5] + __popc(w & (m - 1u));
    return (w & m) != 0 && slot < *n_slots;
}

// Exact 64-bit accumulation (mod 2^64) in shared memory from native 32-bit
// atomics: the low word takes the low half and reports its own wrap-around,
// which is carried into the high word together with the high half.
__device__ __forceinline__ void shared_add64(uint32_t* lo, uint32_t* hi, int c, unsigned long long v) {
    const uint32_t vl = uint32_t(v);
    uint32_t vh = uint32_t(v >> 32);
    const uint32_t old = atomicAdd(&lo[c], vl);
    vh += (old + vl < old) ? 1u : 0u;
    if (vh) atomicAdd(&hi[c], vh);
}

// ---- warp helpers -------------------------------------------------------------
// Lane of the n-th (0-based) member of the lane set `group`, or 32 if the
// group has no more than n members.
__device__ __forceinline__ int nth_member(unsigned group, int n) {
    if (n >= __popc(group)) return 32;
    int pos = 0;  // largest pos with popc(group below pos) <= n
#pragma unroll
    for (int w = 16; w > 0; w >>= 1)
        if (__popc(group & ((1u << (pos + w)) - 1u)) <= n) pos += w;
    return pos;
}

// Sum of v over all 32 lanes of a converged warp, given to every lane.
// Exact modulo 2^64: 16-bit chunks go through the native 32-bit warp
// reduction (a chunk sum over 32 lanes fits in 21 bits).
__device__ __forceinline__ unsigned long long warp_sum64(unsigned long long v) {
    unsigned long long s = 0;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        unsigned c = unsigned((v >> (16 * k)) & 0xffffull);
        s += (unsigned long long)__reduce_add_sync(0xffffffffu, c) << (16 * k);
    }
    return s;
}
__device__ __forceinline__ unsigned long long warp_sum32(unsigned v) {
    return (unsigned long long)__reduce_add_sync(0xffffffffu, v & 0xffffu) +
           ((unsigned long long)__reduce_add_sync(0xffffffffu, v >> 16) << 16);
}

// Sum of v over the lanes of `peers` (lanes sharing one key, as returned by
// __match_any_sync), delivered to the group's lowest lane (rank 0): a
// log-depth tree over the ranks within the group.  All 32 lanes must call it.
template <class T>
__device__ __forceinline__ T group_sum(T v, unsigned peers, int lane, int rank) {
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
        int src = nth_member(peers, rank + s);
        T t = __shfl_sync(0xffffffffu, v, src < 32 ? src : lane);
        if ((rank & (2 * s - 1)) == 0 && src < 32) v += t;
    }
    return v;
}

// ---- host helpers (ctx.cu) --------------------------------------------------
int check_ng(int ng);
int cuda_status(cudaError_t e);
inline void count_launch(cwthf_ctx* c, int n = 1) { c->launches.fetch_add(n, std::memory_order_relaxed); }

// Counts one kernel launch and, when profiling is on, brackets it with CUDA
// events recorded on the launching stream.
struct LaunchScope {
    cwthf_ctx* ctx;
    cudaStream_t s;
    const char* name;
    cudaEvent_t a = nullptr;
    LaunchScope(cwthf_ctx* c, cudaStream_t st, const char* n) : ctx(c), s(st), name(n) {
        count_launch(c);
        if (c->prof_on) {
            a = prof_event(c);
            if (a) cudaEventRecord(a, s);
        }
    }
    ~LaunchScope() {
        if (a) {
            cudaEvent_t b = prof_event(ctx);
            if (b) {
                cudaEventRecord(b, s);
                ctx->prof_pending.push_back({name, a, b});
            }
        }
    }
    static cudaEvent_t prof_event(cwthf_ctx* c) {
        if (!c->prof_pool.empty()) {
            cudaEvent_t e = c->prof_pool.back();
            c->prof_pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        return cudaEventCreate(&e) == cudaSuccess ? e : nullptr;
    }
};
#define CWTHF_LAUNCH(ctx, stream, name, ...)               \
    do {                                                     \
        ::cwthf::LaunchScope _cwthf_scope(ctx, stream, name); \
        __VA_ARGS__;                                         \
    } while (0)

// ---- scan (scan.cu) ----------------------------------------------------------
// Exclusive scan of n uint32 values (n given on the host): out[i] = sum_{j<i} in[j],
// out[n] = total.  in and out may alias.
int scan_u32(cwthf_ctx* ctx, const uint32_t* in, uint32_t* out, int64_t n, cudaStream_t s);
// Same, with the length read from device memory (*d_n <= n_cap).
int scan_u32_dev(cwthf_ctx* ctx, const uint32_t* in, uint32_t* out, const uint32_t* d_n, int64_t n_cap,
                 cudaStream_t s);
size_t scan_tmp_words(int64_t n_cap);

// ---- stages -------------------------------------------------------------------
int deposit_impl(cwthf_ctx* ctx, const float* pos, const float* mass, double mass_unit, int64_t np, double L,
                 int ng, int64_t* grid, int64_t* mtot, cudaStream_t s);
// The binning passes of the deposit alone: packed records per (tile, class)
// in ctx->dep_rec / dep_mq with offsets ctx->dep_off, and sum m_q in d_mtot.
int bin_particles(cwthf_ctx* ctx, const float* pos, const float* mass, double mass_unit, int64_t np, double L, int ng,
                  cudaStream_t s);
// The self-boundness check of every group (Sec. 2.3).
int unbind_impl(cwthf_ctx* ctx, const float* pos, const float* vel, const float* mass, double mass_unit, int64_t np,
                double L, double G, const int32_t* group, int64_t n_groups, int max_iter, int32_t* group_out,
                int64_t* n_kept, int32_t* iters, cudaStream_t s);
// The same with the group count read from device memory (*d_groups <= n_groups).
int unbind_groups(cwthf_ctx* ctx, const float* pos, const float* vel, const float* mass, double mass_unit, int64_t np,
                  double L, double G, const int32_t* group, int64_t n_groups, const uint32_t* d_groups, int max_iter,
                  int32_t* group_out, int64_t* n_kept, int32_t* iters, cudaStream_t s);
// Forward half of the transform: x r2c and y c2c -> ctx spectrum `spec`.
int transform_forward_xy(cwthf_ctx* ctx, const int64_t* grid, int ng, float2* spec, cudaStream_t s);
// The FFT twiddles of ng and the wavelet spectra of the n scales w[] for a box
// of side L, from the context's table slots (wtab[i]: device [2 * ng]).
// Called before anything else of a call is queued.
int transform_tables(cwthf_ctx* ctx, int ng, double L, const double* w, int n, const float** wtab,
                     cudaStream_t s);
// z forward, wavelet multiply with the spectrum wtab, z inverse (src -> dst,
// may alias), then y inverse and x c2r into cwt.
int transform_wavelet_inverse(cwthf_ctx* ctx, float2* src, float2* dst, int ng, double L, double w,
                              double mass_unit, const float* wtab, float* cwt, cudaStream_t s);
int transform_stencil_impl(cwthf_ctx* ctx, const int64_t* grid, int ng, double L, double mass_unit, double w, int R,
                           float* cwt, cudaStream_t s);
int segment_impl(cwthf_ctx* ctx, const float* cwt, int ng, float cwt_min, int32_t* label, bool seeds_ready,
                 cudaStream_t s);
// CTAs of the segmentation fallback's cooperative launch (-1 on failure).
int fallback_blocks(int sm_count);
// CTAs of the self-boundness check's whole-grid launch (-1 on failure).
int unbind_grid_blocks(int sm_count);
// Seeds of the last segmentation and the cell count of each segment.
int segment_sizes_impl(cwthf_ctx* ctx, int32_t* seeds, int64_t* n_cells, int64_t cap, int64_t* n_seeds,
                       cudaStream_t s);
// seeds_ready: the seed bitmap / ranks of `label` are already in ctx (after
// segment_impl); bins_ready: ctx->dep_* hold the binned records of these
// particles for this grid (after deposit_impl).
// scale / n_scales: this call's scale among those of one find; the halo ids
// of all scales are written (halo_id[k * np + i]) once the last one is done.
int assign_impl(cwthf_ctx* ctx, const float* pos, const float* mass, double mass_unit, int64_t np, double L,
                int ng, const int32_t* label, const float* cwt, const cwthf_params* p, int scale, int n_scales,
                int32_t* halo_id, cwthf_halo* cat, int64_t cat_cap, int64_t* n_halo, bool seeds_ready,
                bool bins_ready, cudaStream_t s);
// The multi-scale loop's per-scale pieces (assign.cu): group sums of the
// particles without a halo id at this scale's grid, and their slots (pslot);
// then, one scale later, the keep decision with the cross-scale check against
// the next field Cn (nullptr after the last scale), the catalogue and the ids.
int ms_scale_sums(cwthf_ctx* ctx, const float* pos, const float* mass, double mass_unit, int64_t np, double L, int ng,
                  const int32_t* halo_id, int32_t* pslot, cudaStream_t s);
int ms_finalize(cwthf_ctx* ctx, const float* pos, const float* mass, const float* vel, double G, int max_iter,
                int64_t np, double L, int ng, double mass_unit, const float* C, const float* Cn, int ngn, int scale,
                double dens_th, int64_t particle_th, const int32_t* pslot, const unsigned long long* mtot,
                int32_t* halo_id, cwthf_ms_halo* cat, int64_t cat_cap, int64_t* n_halo, cudaStream_t s);
void free_tables(cwthf_ctx* ctx);
int init_tables(cwthf_ctx* ctx);
// A caller's FFT plan for one pass of grid size ng (fft.cu); nst = 0 clears it.
int set_fft_plan(cwthf_ctx* ctx, int ng, int which, int C, const int* rad, int nst);

// ---- deposit on caller-provided scratch (used by cwthf_deposit_noalloc) ------
struct DepositScratch {
    uint32_t* count;           // [keys + 2]
    uint32_t* off;             // [keys + 2]
    uint32_t* cursor;          // [keys + 2]
    uint32_t* scan_tmp;        // [scan_cap]
    size_t scan_cap;
    unsigned long long* rec;   // [np]
    uint32_t* mq;              // [np]
    unsigned long long* mtot;  // [1]
    int* status;               // [1]
    int sm_count;
};
int deposit_into_scratch(const DepositScratch& sc, const float* pos, const float* mass, double mass_unit, int64_t np,
                         double L, int ng, int64_t* grid, cudaStream_t s);
int scan_u32_scratch(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* tmp, size_t tmp_cap, cudaStream_t s);

}  // namespace cwthf
