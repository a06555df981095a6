// assign.cu -- particles to segments, per-halo sums and thresholds
// (Sec. 2 steps 6-7, Sec. 2.3 centre of mass, Sec. 2.4 and Table 1 density
// and particle thresholds).
//
// Every per-halo sum is an integer: particle count, integer mass sum m_q, and
// the first moment sum m_q * (q - seed * 2^10) of the fixed-point positions
// about the seed node (minimum image), so the catalogue is exact and
// independent of the order of the atomic updates.  Halos are indexed by
// "slot", the rank of their seed among all seeds in cell order, read from the
// seed bitmap and its popcount prefix.
#include "internal.cuh"
#include "quant.cuh"

namespace cwthf {

int seeds_from_labels(cwthf_ctx* ctx, const int32_t* label, int ng, cudaStream_t s);

namespace {

constexpr int kThreads = 256;
constexpr unsigned kFull = 0xffffffffu;
using u64 = unsigned long long;

// Slot of seed cell `lab`; false if lab is not a seed or its slot is beyond
// the number of slots in use.
__device__ __forceinline__ bool seed_slot(const uint32_t* bits, const uint32_t* prefix, const uint32_t* n_slots,
                                          int32_t lab, uint32_t& slot) {
    uint32_t w = bits[lab >> 5];
    uint32_t m = 1u << (lab & 31);
    slot = prefix[lab >> 5] + __popc(w & (m - 1u));
    return (w & m) != 0 && slot < *n_slots;
}

// Cells per seed.
__global__ void __launch_bounds__(kThreads) k_count_cells(const int32_t* __restrict__ label, int64_t cells,
                                                         const uint32_t* __restrict__ bits,
                                                         const uint32_t* __restrict__ prefix,
                                                         const uint32_t* __restrict__ n_slots, HaloAcc* acc,
                                                         int* status) {
    int lane = threadIdx.x & 31;
    int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t base = int64_t(blockIdx.x) * blockDim.x + (threadIdx.x & ~31); base < cells; base += stride) {
        int64_t c = base + lane;
        uint32_t key = 0xffffffffu;
        if (c < cells) {
            int32_t l = label[c];
            uint32_t slot;
            if (l >= 0 && l < cells) {
                if (seed_slot(bits, prefix, n_slots, l, slot)) key = slot;
                else set_status(status, CWTHF_E_BAD_INPUT);
            } else if (l != -1) {
                set_status(status, CWTHF_E_BAD_INPUT);
            }
        }
        unsigned peers = __match_any_sync(kFull, key);
        if (key != 0xffffffffu && lane == __ffs(peers) - 1) atomicAdd(&acc[key].n_cells, u64(__popc(peers)));
    }
}

// Particles: nearest node, its label, slot; integer sums per slot.
__global__ void __launch_bounds__(kThreads) k_assign(DepArgs a, const int32_t* __restrict__ label,
                                                    const uint32_t* __restrict__ bits,
                                                    const uint32_t* __restrict__ prefix,
                                                    const uint32_t* __restrict__ n_slots, HaloAcc* acc,
                                                    int32_t* __restrict__ part_slot, u64* __restrict__ mtot,
                                                    int* status) {
    int lane = threadIdx.x & 31;
    int64_t stride = int64_t(gridDim.x) * blockDim.x;
    const int64_t N = a.ng, M = a.modulus;
    u64 msum = 0;
    for (int64_t base = int64_t(blockIdx.x) * blockDim.x + (threadIdx.x & ~31); base < a.np; base += stride) {
        int64_t i = base + lane;
        uint32_t key = 0xffffffffu;
        uint32_t mq = 0;
        long long mom[3] = {0, 0, 0};
        if (i < a.np) {
            int64_t q[3];
            const float* p = a.pos + 3 * i;
            bool ok = quantise(p[0], a.scale, M, q[0]) && quantise(p[1], a.scale, M, q[1]) &&
                      quantise(p[2], a.scale, M, q[2]);
            int ms = ok ? mass_quantum(a, i, mq) : CWTHF_E_BAD_INPUT;
            int32_t slot_out = -1;
            if (ms != CWTHF_OK) {
                set_status(status, ms);
                mq = 0;
            } else {
                int64_t n[3];
#pragma unroll
                for (int d = 0; d < 3; d++) n[d] = ((q[d] + kFracOne / 2) >> kFracBits) % N;
                int32_t lab = label[(n[2] * N + n[1]) * N + n[0]];
                uint32_t slot;
                if (lab >= 0 && lab < N * N * N && seed_slot(bits, prefix, n_slots, lab, slot)) {
                    key = slot;
                    slot_out = int32_t(slot);
                    int64_t s[3] = {lab % N, (lab / N) % N, lab / (N * N)};
#pragma unroll
                    for (int d = 0; d < 3; d++) {
                        int64_t dq = (q[d] - s[d] * kFracOne) % M;
                        if (dq < 0) dq += M;
                        if (2 * dq >= M) dq -= M;
                        mom[d] = (long long)mq * dq;
                    }
                }
            }
            part_slot[i] = slot_out;
        }
        msum += mq;
        unsigned peers = __match_any_sync(kFull, key);
        int rank = __popc(peers & ((1u << lane) - 1));
        u64 cnt = 1, m_sum = mq;
        long long m0 = mom[0], m1 = mom[1], m2 = mom[2];
        if (__any_sync(kFull, __popc(peers) > 1)) {  // warp-uniform: aggregate groups first
            cnt = __popc(peers);
            m_sum = group_sum<u64>(m_sum, peers, lane, rank);
            m0 = group_sum<long long>(m0, peers, lane, rank);
            m1 = group_sum<long long>(m1, peers, lane, rank);
            m2 = group_sum<long long>(m2, peers, lane, rank);
        }
        if (key != 0xffffffffu && rank == 0) {
            HaloAcc* h = acc + key;
            atomicAdd(&h->n_part, cnt);
            atomicAdd(&h->mq, m_sum);
            atomicAdd(reinterpret_cast<u64*>(&h->mom[0]), u64(m0));
            atomicAdd(reinterpret_cast<u64*>(&h->mom[1]), u64(m1));
            atomicAdd(reinterpret_cast<u64*>(&h->mom[2]), u64(m2));
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) msum += __shfl_xor_sync(kFull, msum, o);
    if (lane == 0 && msum) atomicAdd(mtot, msum);
}

struct FilterArgs {
    int ng;
    double L, mass_unit, dens_th;
    int64_t particle_th;
    int64_t cat_cap;
};

// keep flag per slot (1 / 0), scanned afterwards into output positions.
__global__ void __launch_bounds__(kThreads) k_keep(const HaloAcc* __restrict__ acc, const uint32_t* __restrict__ n_seeds,
                                                  const u64* __restrict__ mtot, FilterArgs f,
                                                  uint32_t* __restrict__ keep) {
    uint32_t ns = *n_seeds;
    double ncube = double(int64_t(f.ng) * f.ng * f.ng);
    double rhs0 = __dmul_rn(f.dens_th, double(*mtot));
    int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < ns; s += stride) {
        HaloAcc h = acc[s];
        bool k = int64_t(h.n_part) >= f.particle_th &&
                 __dmul_rn(double(h.mq), ncube) >= __dmul_rn(rhs0, double(h.n_cells));
        keep[s] = k ? 1u : 0u;
    }
}

__global__ void __launch_bounds__(kThreads) k_catalogue(const HaloAcc* __restrict__ acc,
                                                       const int32_t* __restrict__ seed_list,
                                                       const uint32_t* __restrict__ n_seeds,
                                                       const uint32_t* __restrict__ keep_off, const float* cwt,
                                                       FilterArgs f, cwthf_halo* __restrict__ cat,
                                                       int64_t* __restrict__ n_halo, int* status) {
    uint32_t ns = *n_seeds;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        uint32_t kept = keep_off[ns];
        *n_halo = int64_t(kept);
        if (int64_t(kept) > f.cat_cap) set_status(status, CWTHF_E_CAPACITY);
    }
    const int64_t N = f.ng;
    const double cell_q = (f.L / double(f.ng)) / double(kFracOne);
    int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < ns; s += stride) {
        uint32_t pos = keep_off[s];
        if (keep_off[s + 1] == pos || int64_t(pos) >= f.cat_cap) continue;
        HaloAcc h = acc[s];
        int64_t seed = seed_list[s];
        int64_t sc[3] = {seed % N, (seed / N) % N, seed / (N * N)};
        cwthf_halo o;
        o.seed = seed;
        o.n_part = int64_t(h.n_part);
        o.n_cells = int64_t(h.n_cells);
        o.mass = __dmul_rn(double(h.mq), f.mass_unit);
#pragma unroll
        for (int d = 0; d < 3; d++) {
            double u = double(sc[d] * kFracOne);
            if (h.mq > 0) u = __dadd_rn(u, __ddiv_rn(double(h.mom[d]), double(h.mq)));
            double x = __dmul_rn(u, cell_q);
            if (x >= f.L) x = __dsub_rn(x, f.L);
            else if (x < 0.0) x = __dadd_rn(x, f.L);
            o.centre[d] = x;
        }
        o.peak = cwt ? cwt[seed] : 0.0f;
        o.reserved = 0;
        cat[pos] = o;
    }
}

__global__ void __launch_bounds__(kThreads) k_finalize(const int32_t* __restrict__ part_slot, int64_t np,
                                                      const uint32_t* __restrict__ keep_off,
                                                      const int32_t* __restrict__ seed_list,
                                                      int32_t* __restrict__ halo_id) {
    int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < np; i += stride) {
        int32_t s = part_slot[i];
        int32_t out = -1;
        if (s >= 0 && keep_off[s + 1] != keep_off[s]) out = seed_list[s];
        halo_id[i] = out;
    }
}

}  // namespace

int assign_impl(cwthf_ctx* ctx, const float* pos, const float* mass, double mass_unit, int64_t np, double L, int ng,
                const int32_t* label, const float* cwt, const cwthf_params* p, int32_t* halo_id, cwthf_halo* cat,
                int64_t cat_cap, int64_t* n_halo, bool seeds_ready, cudaStream_t s) {
    int rc;
    if (!seeds_ready && (rc = seeds_from_labels(ctx, label, ng, s))) return rc;
    int64_t cells = int64_t(ng) * ng * ng;
    int64_t nwords = (cells + 31) / 32;
    const uint32_t* d_nseeds = ctx->n_seeds;  // seeds in use (clamped to slot_cap)
    int64_t slot_cap = cells / 8 + 8;
    int blocks = ctx->sm_count * 8;
    cudaError_t e = cudaMemsetAsync(ctx->d_mtot, 0, 8, s);
    if (e != cudaSuccess) return cuda_status(e);
    CWTHF_LAUNCH(ctx, s, "k_count_cells", k_count_cells<<<blocks, kThreads, 0, s>>>(label, cells, ctx->seed_bits, ctx->seed_prefix, d_nseeds, ctx->acc,
                                              ctx->d_status));
    DepArgs a = make_dep_args(pos, mass, mass_unit, np, L, ng);
    int pblocks = int(std::min<int64_t>(div_up(std::max<int64_t>(np, 1), kThreads), int64_t(ctx->sm_count) * 16));
    CWTHF_LAUNCH(ctx, s, "k_assign", k_assign<<<pblocks, kThreads, 0, s>>>(a, label, ctx->seed_bits, ctx->seed_prefix, d_nseeds, ctx->acc, ctx->part_slot,
                                          ctx->d_mtot, ctx->d_status));
    FilterArgs f;
    f.ng = ng;
    f.L = L;
    f.mass_unit = mass_unit;
    f.dens_th = p->dens_th;
    f.particle_th = p->particle_th;
    f.cat_cap = cat_cap;
    CWTHF_LAUNCH(ctx, s, "k_keep", k_keep<<<blocks, kThreads, 0, s>>>(ctx->acc, d_nseeds, ctx->d_mtot, f, ctx->keep_off));
    if ((rc = scan_u32_dev(ctx, ctx->keep_off, ctx->keep_off, d_nseeds, slot_cap, s))) return rc;
    CWTHF_LAUNCH(ctx, s, "k_catalogue", k_catalogue<<<blocks, kThreads, 0, s>>>(ctx->acc, ctx->seed_list, d_nseeds, ctx->keep_off, cwt, f, cat, n_halo,
                                            ctx->d_status));
    CWTHF_LAUNCH(ctx, s, "k_finalize", k_finalize<<<pblocks, kThreads, 0, s>>>(ctx->part_slot, np, ctx->keep_off, ctx->seed_list, halo_id));
    return cuda_status(cudaGetLastError());
}

}  // namespace cwthf
