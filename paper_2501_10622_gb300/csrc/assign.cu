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

// Cells per seed: four labels per thread and iteration, one atomic per slot
// per warp.
__global__ void __launch_bounds__(kThreads) k_count_cells(const int32_t* __restrict__ label, int64_t cells,
                                                         const uint32_t* __restrict__ bits,
                                                         const uint32_t* __restrict__ prefix,
                                                         const uint32_t* __restrict__ n_slots, HaloAcc* acc,
                                                         int* status) {
    const int lane = threadIdx.x & 31;
    const int64_t n4 = (cells + 3) / 4;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t base = int64_t(blockIdx.x) * blockDim.x + (threadIdx.x & ~31); base < n4; base += stride) {
        const int64_t i = base + lane;  // warp-uniform trip count
        int l[4] = {-1, -1, -1, -1};
        if (i < n4) {
            if (4 * i + 3 < cells) {
                const int4 q = reinterpret_cast<const int4*>(label)[i];
                l[0] = q.x; l[1] = q.y; l[2] = q.z; l[3] = q.w;
            } else {
                for (int j = 0; j < 4 && 4 * i + j < cells; j++) l[j] = label[4 * i + j];
            }
        }
#pragma unroll
        for (int j = 0; j < 4; j++) {
            uint32_t key = 0xffffffffu;
            if (l[j] >= 0 && l[j] < cells) {
                uint32_t slot;
                if (seed_slot(bits, prefix, n_slots, l[j], slot)) key = slot;
                else set_status(status, CWTHF_E_BAD_INPUT);
            } else if (l[j] != -1) {
                set_status(status, CWTHF_E_BAD_INPUT);
            }
            const unsigned peers = __match_any_sync(kFull, key);
            if (key != 0xffffffffu && lane == __ffs(peers) - 1) atomicAdd(&acc[key].n_cells, u64(__popc(peers)));
        }
    }
}

// Nearest node per axis from the fixed-point coordinate q in [0, ng*2^10):
// (q + 2^9) >> 10, with ng wrapping to 0.
__device__ __forceinline__ int nearest_node(int64_t q, int ng) {
    int n = int((q + kFracOne / 2) >> kFracBits);
    return n == ng ? 0 : n;
}

// Quotient by the grid size without a divide instruction: with
// m = ceil(2^64 / d), the high word of n * m is floor(n / d) for every 32-bit
// n and 2 <= d < 2^32 (n * m / 2^64 exceeds n / d by less than n / 2^64 < 1/d,
// which cannot reach the next integer).
struct FastDiv {
    unsigned long long m;
    uint32_t d;
};
inline FastDiv make_fastdiv(uint32_t d) { return {~0ull / d + 1ull, d}; }
__device__ __forceinline__ uint32_t fdiv(uint32_t n, FastDiv f) { return uint32_t(__umul64hi((unsigned long long)n, f.m)); }

// Per-halo integer sums over the binned records.  A CTA takes kChunk
// consecutive records at a time (records are grouped by deposit tile, a
// 32 x 8 x 8-cell block, so a chunk covers a few neighbouring tiles and a
// few dozen halos), kRecPerThread per thread with independent gather chains
// (record -> label -> seed bitmap and prefix).  The chunk is first folded into
// a small open-addressing table of halo slots in shared memory, then each
// table entry is added to the global accumulators once; a record whose slot
// finds no entry within kProbe probes goes straight to the global atomics.  A
// warp whose 32 records share one halo is folded with warp reductions first.
// Each record's halo slot (or -1) is kept for the final pass, at
// rec_slot[r * slot_stride].
//
// Equal masses (kMass false): a record's moment is its offset dq from the
// seed, |dq| < ng 2^9 <= 2^20, so a chunk's sum per entry stays below 2^30 and
// the table holds plain 32-bit integers.  Per-particle masses: products
// m_q dq need 64 bits, kept exactly as two 32-bit words with the carry.
constexpr int kHsThreads = 256;
// resident CTAs per SM: registers (equal masses) or the 45 KB table (masses)
template <bool kMass> constexpr int hs_ctas_per_sm() { return kMass ? 4 : 6; }
constexpr int kTabBits = 10, kTab = 1 << kTabBits;  // table entries per CTA
constexpr int kProbe = 16;
constexpr int kRecPerThread = 4;
constexpr int kChunk = kHsThreads * kRecPerThread;
constexpr uint32_t kEmpty = 0xffffffffu;
static_assert(int64_t(kChunk) * (int64_t(CWTHF_MAX_NG) << (CWTHF_FRAC_BITS - 1)) < (int64_t(1) << 31),
              "a chunk's equal-mass moment sums must fit 32 bits");

__device__ __forceinline__ void global_halo_add(HaloAcc* h, u64 cnt, u64 mq, u64 m0, u64 m1, u64 m2) {
    atomicAdd(&h->n_part, cnt);
    atomicAdd(&h->mq, mq);
    atomicAdd(reinterpret_cast<u64*>(&h->mom[0]), m0);
    atomicAdd(reinterpret_cast<u64*>(&h->mom[1]), m1);
    atomicAdd(reinterpret_cast<u64*>(&h->mom[2]), m2);
}

// A 32-bit two's-complement sum as the 64-bit word the accumulators add.
__device__ __forceinline__ u64 sext(uint32_t v) { return u64((long long)int32_t(v)); }
__device__ __forceinline__ u64 sext(int32_t v) { return u64((long long)v); }

// The table entry of halo slot `key`: found, or claimed (and listed in tused)
// when an empty entry comes first; -1 after kProbe probes.
__device__ __forceinline__ int table_find(uint32_t* tkey, uint32_t* tused, uint32_t* used, uint32_t key) {
    uint32_t h = (key * 2654435761u) >> (32 - kTabBits);  // multiplicative hash
    for (int pr = 0; pr < kProbe; pr++, h = (h + 1) & (kTab - 1)) {
        uint32_t k = tkey[h];
        if (k == kEmpty) {
            k = atomicCAS(&tkey[h], kEmpty, key);
            if (k == kEmpty) {
                tused[atomicAdd(used, 1u)] = h;
                return int(h);
            }
        }
        if (k == key) return int(h);
    }
    return -1;
}

template <bool kMass>
__global__ void __launch_bounds__(kHsThreads, hs_ctas_per_sm<kMass>()) k_halo_sums(DepArgs a, FastDiv divn, const uint32_t* __restrict__ total_ptr,
                                                       const unsigned long long* __restrict__ rec,
                                                       const uint32_t* __restrict__ rec_mq,
                                                       const int32_t* __restrict__ label,
                                                       const uint32_t* __restrict__ bits,
                                                       const uint32_t* __restrict__ prefix,
                                                       const uint32_t* __restrict__ n_slots, HaloAcc* acc,
                                                       int32_t* __restrict__ rec_slot, int slot_stride,
                                                       u64* __restrict__ mtot, int skip_marked, int* status) {
    constexpr int kW = kMass ? kTab : 1;  // the 64-bit words exist with masses only
    __shared__ uint32_t tkey[kTab], tcnt[kTab], tused[kTab];
    __shared__ uint32_t tm_lo[3][kTab];  // moments (equal masses: the whole 32-bit sum)
    __shared__ uint32_t tm_hi[3][kW], tmq_lo[kW], tmq_hi[kW];
    __shared__ uint32_t n_used[2];
    const int lane = threadIdx.x & 31;
    const int N = a.ng;
    const int32_t M = int32_t(a.modulus);
    const int64_t cells = int64_t(N) * N * N;
    const int64_t total = *total_ptr;  // records binned
    const uint32_t ns = *n_slots;
    for (int e = threadIdx.x; e < kTab; e += blockDim.x) {
        tkey[e] = kEmpty;
        tcnt[e] = 0u;
        tm_lo[0][e] = tm_lo[1][e] = tm_lo[2][e] = 0u;
        if (kMass) {
            tmq_lo[e] = tmq_hi[e] = 0u;
            tm_hi[0][e] = tm_hi[1][e] = tm_hi[2][e] = 0u;
        }
    }
    if (threadIdx.x < 2) n_used[threadIdx.x] = 0;
    __syncthreads();
    u64 msum = 0;
    int it = 0;
    for (int64_t c0 = int64_t(blockIdx.x) * kChunk; c0 < total; c0 += int64_t(gridDim.x) * kChunk, it ^= 1) {
        uint32_t* used = &n_used[it];
        // gathers for kRecPerThread records, warp-contiguous runs of 32
        u64 e[kRecPerThread];
        uint32_t mq[kRecPerThread];
        int32_t lab[kRecPerThread];
#pragma unroll
        for (int u = 0; u < kRecPerThread; u++) {
            const int64_t r = c0 + u * kHsThreads + threadIdx.x;
            mq[u] = 0;
            lab[u] = -1;
            e[u] = 0;
            if (r < total) {
                e[u] = rec[r];
                mq[u] = kMass ? rec_mq[r] : 1u;
                // a record marked in bit 63 (its particle already holds a halo id)
                // joins no group
                if (!(skip_marked && (e[u] >> 63))) {
                    const int64_t node = (int64_t(nearest_node(rec_q(e[u], 2), N)) * N +
                                          nearest_node(rec_q(e[u], 1), N)) * N + nearest_node(rec_q(e[u], 0), N);
                    if (index_ok(node, cells, status)) lab[u] = label[node];
                }
            }
        }
        uint32_t word[kRecPerThread], pre[kRecPerThread];
#pragma unroll
        for (int u = 0; u < kRecPerThread; u++) {
            const bool in = lab[u] >= 0 && int64_t(lab[u]) < cells;
            word[u] = in ? bits[lab[u] >> 5] : 0u;
            pre[u] = in ? prefix[lab[u] >> 5] : 0u;
        }
#pragma unroll
        for (int u = 0; u < kRecPerThread; u++) {
            const int64_t r = c0 + u * kHsThreads + threadIdx.x;
            uint32_t key = kEmpty;
            int32_t dq[3] = {0, 0, 0};
            if (r < total) {
                const uint32_t bit = 1u << (lab[u] & 31);
                const uint32_t slot = pre[u] + __popc(word[u] & (bit - 1u));
                if ((word[u] & bit) && slot < ns) {
                    key = slot;
                    const uint32_t t = fdiv(uint32_t(lab[u]), divn), z = fdiv(t, divn);
                    const int32_t sc[3] = {int32_t(uint32_t(lab[u]) - t * divn.d), int32_t(t - z * divn.d), int32_t(z)};
#pragma unroll
                    for (int d = 0; d < 3; d++) {
                        int32_t v = rec_q(e[u], d) - (sc[d] << kFracBits);  // in (-M, M)
                        if (v < 0) v += M;
                        if (2 * v >= M) v -= M;  // minimum image in [-M/2, M/2)
                        dq[d] = v;
                    }
                }
                rec_slot[r * slot_stride] = int32_t(key);  // kEmpty reads as -1
            }
            msum += mq[u];
            // all 32 records in one halo: one lane carries the warp's sums (the
            // shuffle runs on every lane)
            const uint32_t k0 = __shfl_sync(kFull, key, 0);
            const bool uniform = __all_sync(kFull, key == k0) && key != kEmpty;
            if (kMass) {
                u64 cnt = 1, m_sum = mq[u];
                u64 m[3];
#pragma unroll
                for (int d = 0; d < 3; d++) m[d] = u64((long long)mq[u] * dq[d]);
                if (uniform) {
                    cnt = 32;
                    m_sum = warp_sum32(mq[u]);
#pragma unroll
                    for (int d = 0; d < 3; d++) m[d] = warp_sum64(m[d]);
                }
                if (key != kEmpty && (!uniform || lane == 0)) {
                    const int f = table_find(tkey, tused, used, key);
                    if (f >= 0) {
                        atomicAdd(&tcnt[f], uint32_t(cnt));
                        shared_add64(tmq_lo, tmq_hi, f, m_sum);
#pragma unroll
                        for (int d = 0; d < 3; d++) shared_add64(tm_lo[d], tm_hi[d], f, m[d]);
                    } else {
                        global_halo_add(acc + key, cnt, m_sum, m[0], m[1], m[2]);
                    }
                }
            } else {
                uint32_t cnt = 1;
                int32_t m[3] = {dq[0], dq[1], dq[2]};
                if (uniform) {
                    cnt = 32;
#pragma unroll
                    for (int d = 0; d < 3; d++) m[d] = __reduce_add_sync(kFull, m[d]);
                }
                if (key != kEmpty && (!uniform || lane == 0)) {
                    const int f = table_find(tkey, tused, used, key);
                    if (f >= 0) {
                        atomicAdd(&tcnt[f], cnt);
#pragma unroll
                        for (int d = 0; d < 3; d++) atomicAdd(reinterpret_cast<int*>(&tm_lo[d][f]), m[d]);
                    } else {
                        global_halo_add(acc + key, cnt, cnt, sext(m[0]), sext(m[1]),
                                        sext(m[2]));
                    }
                }
            }
        }
        __syncthreads();
        // one set of global atomics per table entry used by this chunk; the entries are
        // cleared, and the other counter is reset for the next chunk (its last readers
        // passed the barrier above)
        const uint32_t nu = *used;
        if (threadIdx.x == 0) n_used[it ^ 1] = 0;
        for (uint32_t j = threadIdx.x; j < nu; j += blockDim.x) {
            const uint32_t h = tused[j];
            const u64 c = tcnt[h];
            if (kMass) {
                global_halo_add(acc + tkey[h], c, (u64(tmq_hi[h]) << 32) | tmq_lo[h],
                                (u64(tm_hi[0][h]) << 32) | tm_lo[0][h], (u64(tm_hi[1][h]) << 32) | tm_lo[1][h],
                                (u64(tm_hi[2][h]) << 32) | tm_lo[2][h]);
                tmq_lo[h] = tmq_hi[h] = 0u;
                tm_hi[0][h] = tm_hi[1][h] = tm_hi[2][h] = 0u;
            } else {  // the 32-bit sums sign-extended to the 64-bit accumulators
                global_halo_add(acc + tkey[h], c, c, sext(tm_lo[0][h]),
                                sext(tm_lo[1][h]), sext(tm_lo[2][h]));
            }
            tkey[h] = kEmpty;
            tcnt[h] = 0u;
            tm_lo[0][h] = tm_lo[1][h] = tm_lo[2][h] = 0u;
        }
        __syncthreads();
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) msum += __shfl_xor_sync(kFull, msum, o);
    if (lane == 0 && msum) atomicAdd(mtot, msum);
}

// Launches the equal-mass or the per-particle-mass form of k_halo_sums: one
// wave of resident CTAs (fewer for small inputs) striding over the chunks.
void launch_halo_sums(cwthf_ctx* ctx, cudaStream_t s, int64_t np, const DepArgs& a, const uint32_t* total,
                      const unsigned long long* rec, const uint32_t* rec_mq, const int32_t* label,
                      const uint32_t* bits, const uint32_t* prefix, const uint32_t* n_slots, HaloAcc* acc,
                      int32_t* rec_slot, int slot_stride, u64* mtot, int skip_marked) {
    int* st = ctx->d_status;
    const FastDiv dn = make_fastdiv(uint32_t(a.ng));
    const int64_t chunks = div_up(std::max<int64_t>(np, 1), kChunk);
    if (a.mass)
        CWTHF_LAUNCH(ctx, s, "k_halo_sums",
                     k_halo_sums<true><<<int(std::min<int64_t>(chunks, int64_t(ctx->sm_count) * hs_ctas_per_sm<true>())),
                                         kHsThreads, 0, s>>>(a, dn, total, rec, rec_mq, label, bits, prefix, n_slots,
                                                             acc, rec_slot, slot_stride, mtot, skip_marked, st));
    else
        CWTHF_LAUNCH(ctx, s, "k_halo_sums",
                     k_halo_sums<false><<<int(std::min<int64_t>(chunks, int64_t(ctx->sm_count) * hs_ctas_per_sm<false>())),
                                          kHsThreads, 0, s>>>(a, dn, total, rec, rec_mq, label, bits, prefix, n_slots,
                                                              acc, rec_slot, slot_stride, mtot, skip_marked, st));
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
                                                       int32_t* __restrict__ slot_halo,
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
        const uint32_t pos = keep_off[s];
        const bool kept = keep_off[s + 1] != pos;
        slot_halo[s] = kept ? seed_list[s] : -1;
        if (!kept || int64_t(pos) >= f.cat_cap) continue;
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

// Each scale's pass stores its record slots contiguously (rec_slot[scale * np
// + r]: whole sectors written, none read back).  After the last scale the halo
// ids are regrouped per record, RS ids per record (one scale: in place; two:
// 8-byte groups; more: 16-byte groups of four scales), so that the final pass
// reads a particle's ids with one vector gather per four scales.
__host__ __device__ __forceinline__ int slot_group_stride(int n_scales) {
    return n_scales <= 2 ? n_scales : (n_scales + 3) & ~3;
}
__host__ __device__ __forceinline__ int64_t slot_groups_offset(int n_scales, int64_t np) {
    return n_scales == 1 ? 0 : (int64_t(n_scales) * np + 3) & ~int64_t(3);
}

template <int RS>
struct IdGroup;
template <>
struct IdGroup<1> {
    using T = int32_t;
    __device__ static T make(const int32_t* v) { return v[0]; }
    __device__ static int32_t get(const T& g, int j) { return g; }
    __device__ static T none() { return -1; }
};
template <>
struct IdGroup<2> {
    using T = int2;
    __device__ static T make(const int32_t* v) { return make_int2(v[0], v[1]); }
    __device__ static int32_t get(const T& g, int j) { return j == 0 ? g.x : g.y; }
    __device__ static T none() { return make_int2(-1, -1); }
};
template <>
struct IdGroup<4> {
    using T = int4;
    __device__ static T make(const int32_t* v) { return make_int4(v[0], v[1], v[2], v[3]); }
    __device__ static int32_t get(const T& g, int j) { return j == 0 ? g.x : (j == 1 ? g.y : (j == 2 ? g.z : g.w)); }
    __device__ static T none() { return make_int4(-1, -1, -1, -1); }
};

// Record order, after the last scale: each record's slot of every scale becomes
// its halo id (the slot's seed if the halo was kept, else -1), written to the
// record's group (RS = 4: one group per four scales).  Records are grouped by
// tile, so the slot lookups are coherent.  With one scale the groups are the
// slots themselves (each thread rewrites its own entry).
template <int RS>
__global__ void __launch_bounds__(kThreads) k_rec_halo(const int32_t* rec_slot, int64_t np,
                                                      const uint32_t* __restrict__ total_ptr, int n_scales,
                                                      const int32_t* __restrict__ slot_halo, int64_t slot_stride,
                                                      typename IdGroup<RS>::T* groups) {
    constexpr int G = RS < 4 ? RS : 4;  // ids per stored group
    const int64_t total = *total_ptr;
    const int ngr = (n_scales + G - 1) / G;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < total; r += stride) {
        for (int g = 0; g < ngr; g++) {
            int32_t v[G];
#pragma unroll
            for (int j = 0; j < G; j++) {
                const int k = G * g + j;
                const int32_t sl = k < n_scales ? rec_slot[k * np + r] : -1;
                v[j] = sl >= 0 ? slot_halo[k * slot_stride + sl] : -1;
            }
            groups[r * ngr + g] = IdGroup<RS>::make(v);
        }
    }
}

// halo_id of every particle for every scale, in particle order: one gather
// per particle and group of its record's ids.  Several particles per thread
// keep independent gathers in flight.
template <int RS>
__global__ void __launch_bounds__(kThreads) k_finalize(const uint32_t* __restrict__ part_rec, int64_t np,
                                                      const uint32_t* __restrict__ total_ptr,
                                                      const typename IdGroup<RS>::T* __restrict__ groups,
                                                      int n_scales, int32_t* __restrict__ halo_id) {
    constexpr int kIlp = 8;
    constexpr int G = RS < 4 ? RS : 4;
    using T = typename IdGroup<RS>::T;
    const int64_t total = *total_ptr;
    const int ngr = (n_scales + G - 1) / G;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i0 = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i0 < np; i0 += kIlp * stride) {
        int64_t r[kIlp];
#pragma unroll
        for (int u = 0; u < kIlp; u++) {
            const int64_t i = i0 + u * stride;
            const uint32_t x = i < np ? part_rec[i] : 0xffffffffu;
            r[u] = int64_t(x) < total ? int64_t(x) : -1;
        }
        for (int g = 0; g < ngr; g++) {
            T h[kIlp];
#pragma unroll
            for (int u = 0; u < kIlp; u++) h[u] = r[u] >= 0 ? groups[r[u] * ngr + g] : IdGroup<RS>::none();
#pragma unroll
            for (int u = 0; u < kIlp; u++) {
                const int64_t i = i0 + u * stride;
                if (i >= np) continue;
#pragma unroll
                for (int j = 0; j < G; j++)
                    if (G * g + j < n_scales) halo_id[(G * g + j) * np + i] = IdGroup<RS>::get(h[u], j);
            }
        }
    }
}

template <int RS>
void launch_ids(cwthf_ctx* ctx, cudaStream_t s, int blocks, int pblocks, int64_t np, const uint32_t* total,
                int n_scales, int64_t slot_cap, int32_t* halo_id) {
    using T = typename IdGroup<RS>::T;
    T* groups = reinterpret_cast<T*>(ctx->part_slot + slot_groups_offset(n_scales, np));
    CWTHF_LAUNCH(ctx, s, "k_rec_halo",
                 k_rec_halo<RS><<<blocks, kThreads, 0, s>>>(ctx->part_slot, np, total, n_scales, ctx->slot_halo,
                                                            slot_cap, groups));
    CWTHF_LAUNCH(ctx, s, "k_finalize",
                 k_finalize<RS><<<pblocks, kThreads, 0, s>>>(ctx->part_rec, np, total, groups, n_scales, halo_id));
}

// ---- the multi-scale loop (Sec. 2, Fig. 1; App. B; Sec. 2.4) -----------------

// Records of particles that already hold a halo id are marked in bit 63, so
// that this scale's group sums skip them (Sec. 2 step 6: only particles
// without a halo id are assigned).
__global__ void __launch_bounds__(kThreads) k_ms_mark(const int32_t* __restrict__ halo_id,
                                                     const uint32_t* __restrict__ part_rec, int64_t np,
                                                     const uint32_t* __restrict__ total_ptr,
                                                     unsigned long long* __restrict__ rec) {
    const int64_t total = *total_ptr;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < np; i += stride) {
        const uint32_t r = part_rec[i];
        if (halo_id[i] >= 0 && int64_t(r) < total) rec[r] |= 1ull << 63;
    }
}

// Each particle's group slot at this scale (-1: in no group), kept until the
// scale's halos are decided one iteration later.
__global__ void __launch_bounds__(kThreads) k_ms_pslot(const uint32_t* __restrict__ part_rec, int64_t np,
                                                      const uint32_t* __restrict__ total_ptr,
                                                      const int32_t* __restrict__ rec_slot, int32_t* __restrict__ pslot) {
    const int64_t total = *total_ptr;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < np; i += stride) {
        const uint32_t r = part_rec[i];
        pslot[i] = int64_t(r) < total ? rec_slot[r] : -1;
    }
}

// App. B, Eq. B1 along one axis: A the higher and C the lower neighbour of the
// maximum B; l1 = v_A - v_C, l2 = v_B - v_C; the quadratic through A, B, C
// peaks l1^2 / (16 l2 - 8 l1) above B.  Single precision, every operation
// rounded on its own (no contraction), in a fixed order.
__device__ __forceinline__ float ms_peak_term(float vm, float vb, float vp, float& l1, float& l2) {
    const float va = vm > vp ? vm : vp, vc = vm > vp ? vp : vm;
    l1 = __fsub_rn(va, vc);
    l2 = __fsub_rn(vb, vc);
    const float den = __fsub_rn(__fmul_rn(16.0f, l2), __fmul_rn(8.0f, l1));
    return den > 0.0f ? __fdiv_rn(__fmul_rn(l1, l1), den) : 0.0f;
}

// The corrected peak of the maximum at node s (App. B): the node value plus
// the x, y and z terms of Eq. B1, plus, when the next scale's grid has ngn
// nodes per side, the grid-size term (5/16)(2 mean l2 - mean l1)(1 - (ng/ngn)^2).
__device__ float ms_corrected_peak(const float* __restrict__ C, int ng, int64_t s, int ngn) {
    const int64_t n = ng, x = s % n, y = (s / n) % n, z = s / (n * n);
    const int64_t xm = (x + n - 1) % n, xp = (x + 1) % n, ym = (y + n - 1) % n, yp = (y + 1) % n;
    const int64_t zm = (z + n - 1) % n, zp = (z + 1) % n;
    const float vb = C[s];
    float l1x, l2x, l1y, l2y, l1z, l2z;
    const float tx = ms_peak_term(C[(z * n + y) * n + xm], vb, C[(z * n + y) * n + xp], l1x, l2x);
    const float ty = ms_peak_term(C[(z * n + ym) * n + x], vb, C[(z * n + yp) * n + x], l1y, l2y);
    const float tz = ms_peak_term(C[(zm * n + y) * n + x], vb, C[(zp * n + y) * n + x], l1z, l2z);
    float p = __fadd_rn(__fadd_rn(__fadd_rn(vb, tx), ty), tz);
    if (ngn > 0) {
        const float r = __fdiv_rn(float(ng), float(ngn));
        const float m1 = __fdiv_rn(__fadd_rn(__fadd_rn(l1x, l1y), l1z), 3.0f);
        const float m2 = __fdiv_rn(__fadd_rn(__fadd_rn(l2x, l2y), l2z), 3.0f);
        p = __fadd_rn(p, __fmul_rn(__fmul_rn(0.3125f, __fsub_rn(__fmul_rn(2.0f, m2), m1)),
                                   __fsub_rn(1.0f, __fmul_rn(r, r))));
    }
    return p;
}

// Sec. 2 (Fig. 1): a maximum is kept as a maximum in 4D iff its corrected peak
// exceeds every node of the next scale's field enclosing its position (the
// 2 x 2 x 2 nodes around s * L / ng), or 0 after the last scale.
__device__ bool ms_cross_scale(const float* __restrict__ C, int ng, int64_t s, const float* __restrict__ Cn,
                               int ngn, float& peak) {
    peak = ms_corrected_peak(C, ng, s, Cn ? ngn : 0);
    if (!Cn) return peak > 0.0f;
    const int64_t c[3] = {s % ng, (s / ng) % ng, s / (int64_t(ng) * ng)};
    int64_t lo[3], hi[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        lo[a] = (c[a] * ngn) / ng;
        hi[a] = (lo[a] + 1) % ngn;
    }
    const int64_t m = ngn;
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 8; k++) {
        const int64_t gx = (k & 1) ? hi[0] : lo[0], gy = (k & 2) ? hi[1] : lo[1], gz = (k & 4) ? hi[2] : lo[2];
        ok &= peak > Cn[(gz * m + gy) * m + gx];
    }
    return ok;
}

// Keep flag per group (slot): particle and density thresholds (same operands
// as the single-scale path) and the cross-scale check.
__global__ void __launch_bounds__(kThreads) k_ms_keep(const HaloAcc* __restrict__ acc,
                                                     const int32_t* __restrict__ seed_list,
                                                     const uint32_t* __restrict__ n_seeds,
                                                     const u64* __restrict__ mtot, FilterArgs f,
                                                     const float* __restrict__ C, const float* __restrict__ Cn,
                                                     int ngn, uint32_t* __restrict__ keep) {
    const uint32_t ns = *n_seeds;
    const double ncube = double(int64_t(f.ng) * f.ng * f.ng);
    const double rhs0 = __dmul_rn(f.dens_th, double(*mtot));
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < ns; s += stride) {
        const HaloAcc h = acc[s];
        float peak;
        const bool k = int64_t(h.n_part) >= f.particle_th &&
                       __dmul_rn(double(h.mq), ncube) >= __dmul_rn(rhs0, double(h.n_cells)) &&
                       ms_cross_scale(C, f.ng, seed_list[s], Cn, ngn, peak);
        keep[s] = k ? 1u : 0u;
    }
}

// Kept groups become halos base + rank (base: halos of the earlier scales, read
// from *n_halo); catalogue entries, and each slot's halo id (-1: not kept).
__global__ void __launch_bounds__(kThreads) k_ms_catalogue(const HaloAcc* __restrict__ acc,
                                                          const int32_t* __restrict__ seed_list,
                                                          const uint32_t* __restrict__ n_seeds,
                                                          const uint32_t* __restrict__ keep_off, FilterArgs f,
                                                          const float* __restrict__ C, const float* __restrict__ Cn,
                                                          int ngn, int scale, const int64_t* __restrict__ n_halo,
                                                          cwthf_ms_halo* __restrict__ cat,
                                                          int32_t* __restrict__ slot_halo) {
    const uint32_t ns = *n_seeds;
    const int64_t base = *n_halo;
    const int64_t N = f.ng;
    const double cell_q = (f.L / double(f.ng)) / double(kFracOne);
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < ns; s += stride) {
        const uint32_t rank = keep_off[s];
        const bool kept = keep_off[s + 1] != rank;
        const int64_t id = base + rank;
        slot_halo[s] = kept ? int32_t(id) : -1;
        if (!kept || id >= f.cat_cap) continue;
        const HaloAcc h = acc[s];
        const int64_t seed = seed_list[s];
        const int64_t sc[3] = {seed % N, (seed / N) % N, seed / (N * N)};
        cwthf_ms_halo o;
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
        o.peak = ms_corrected_peak(C, f.ng, seed, Cn ? ngn : 0);
        o.scale = scale;
        cat[id] = o;
    }
}

// The number of kept groups (keep_off[n_seeds]) as the check's group count.
__global__ void k_ms_ub_count(const uint32_t* __restrict__ keep_off, const uint32_t* __restrict__ n_seeds,
                              uint32_t* __restrict__ n_groups) {
    *n_groups = keep_off[*n_seeds];
}

// The self-boundness check inside the loop (Sec. 2 step 9, Sec. 2.3): the
// group of each candidate particle of a kept group (its rank among the kept
// groups), or -1.
__global__ void __launch_bounds__(kThreads) k_ms_ub_group(const int32_t* __restrict__ pslot,
                                                         const int32_t* __restrict__ halo_id, int64_t np,
                                                         const uint32_t* __restrict__ keep_off,
                                                         int32_t* __restrict__ grp) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < np; i += stride) {
        const int32_t sl = pslot[i];
        int32_t g = -1;
        if (sl >= 0 && halo_id[i] < 0) {
            const uint32_t r = keep_off[sl];
            if (keep_off[sl + 1] != r) g = int32_t(r);
        }
        grp[i] = g;
    }
}

// Kept groups that the check did not discard stay (flag per slot, scanned
// into their ranks afterwards); their particle count, mass and first moment
// are cleared, to be summed again over the members that stay.
__global__ void __launch_bounds__(kThreads) k_ms_ub_keep(const uint32_t* __restrict__ n_seeds,
                                                        const uint32_t* __restrict__ keep_off,
                                                        const int64_t* __restrict__ n_kept, HaloAcc* acc,
                                                        uint32_t* __restrict__ keep2) {
    const uint32_t ns = *n_seeds;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < ns; s += stride) {
        const uint32_t r = keep_off[s];
        const bool kept = keep_off[s + 1] != r;
        keep2[s] = (kept && n_kept[r] > 0) ? 1u : 0u;
        if (kept) {
            acc[s].n_part = 0;
            acc[s].mq = 0;
            acc[s].mom[0] = acc[s].mom[1] = acc[s].mom[2] = 0;
        }
    }
}

// The sums of the members that stay (bound[i] >= 0): count, integer mass and
// first moment about the seed node, with the group sums' fixed-point rule on
// this scale's grid.
__global__ void __launch_bounds__(kThreads) k_ms_ub_sums(DepArgs a, const int32_t* __restrict__ pslot,
                                                        const int32_t* __restrict__ bound,
                                                        const int32_t* __restrict__ seed_list, HaloAcc* acc) {
    const int N = a.ng;
    const int64_t M = a.modulus;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < a.np; i += stride) {
        if (bound[i] < 0) continue;
        const int32_t sl = pslot[i];
        int64_t q[3];
        uint32_t mq;
        const float* p = a.pos + 3 * i;
        if (!quantise(p[0], a.scale_m, a.scale_e, M, q[0]) || !quantise(p[1], a.scale_m, a.scale_e, M, q[1]) ||
            !quantise(p[2], a.scale_m, a.scale_e, M, q[2]) || mass_quantum(a, i, mq) != CWTHF_OK)
            continue;  // (reported by the deposit of this scale)
        const int32_t seed = seed_list[sl];
        const int sc[3] = {seed % N, (seed / N) % N, seed / (N * N)};
        HaloAcc* h = acc + sl;
        atomicAdd(&h->n_part, 1ull);
        atomicAdd(&h->mq, (u64)mq);
#pragma unroll
        for (int d = 0; d < 3; d++) {
            int64_t dq = q[d] - int64_t(sc[d]) * kFracOne;
            if (dq < 0) dq += M;
            if (2 * dq >= M) dq -= M;  // minimum image in [-M/2, M/2)
            atomicAdd(reinterpret_cast<u64*>(&h->mom[d]), u64((long long)mq * dq));
        }
    }
}

// Particles without a halo id whose group was kept take the halo's id (with
// the self-boundness check: only the members that stayed).
__global__ void __launch_bounds__(kThreads) k_ms_ids(const int32_t* __restrict__ pslot, int64_t np,
                                                    const int32_t* __restrict__ slot_halo,
                                                    const int32_t* __restrict__ bound, int32_t* __restrict__ halo_id) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < np; i += stride) {
        const int32_t sl = pslot[i];
        if (sl >= 0 && halo_id[i] < 0 && (!bound || bound[i] >= 0)) {
            const int32_t id = slot_halo[sl];
            if (id >= 0) halo_id[i] = id;
        }
    }
}

// The running halo count after a scale: n_halo += kept groups; more halos
// than cat_cap is reported as CWTHF_E_CAPACITY (the count is still exact).
__global__ void k_ms_advance(const uint32_t* __restrict__ keep_off, const uint32_t* __restrict__ n_seeds,
                             int64_t* __restrict__ n_halo, int64_t cat_cap, int* status) {
    const int64_t n = *n_halo + int64_t(keep_off[*n_seeds]);
    *n_halo = n;
    if (n > cat_cap) set_status(status, CWTHF_E_CAPACITY);
}

}  // namespace

int ms_scale_sums(cwthf_ctx* ctx, const float* pos, const float* mass, double mass_unit, int64_t np, double L, int ng,
                  const int32_t* halo_id, int32_t* pslot, cudaStream_t s) {
    const int64_t total_key = deposit_geom(ng).ntiles * kDepClasses;
    const uint32_t* total = ctx->dep_off + total_key;
    const int pblocks = int(std::min<int64_t>(div_up(std::max<int64_t>(np, 1), kThreads), int64_t(ctx->sm_count) * 16));
    CWTHF_LAUNCH(ctx, s, "k_ms_mark", k_ms_mark<<<pblocks, kThreads, 0, s>>>(halo_id, ctx->part_rec, np, total, ctx->dep_rec));
    DepArgs a = make_dep_args(pos, mass, mass_unit, np, L, ng);
    int32_t* rec_slot = ctx->part_slot;
    launch_halo_sums(ctx, s, np, a, total, ctx->dep_rec, ctx->dep_mq, ctx->label, ctx->seed_bits,
                     ctx->seed_prefix, ctx->n_seeds, ctx->acc, rec_slot, 1, ctx->d_mtot, 1);
    CWTHF_LAUNCH(ctx, s, "k_ms_pslot", k_ms_pslot<<<pblocks, kThreads, 0, s>>>(ctx->part_rec, np, total, rec_slot, pslot));
    return cuda_status(cudaGetLastError());
}

int ms_finalize(cwthf_ctx* ctx, const float* pos, const float* mass, const float* vel, double G, int max_iter,
                int64_t np, double L, int ng, double mass_unit, const float* C, const float* Cn, int ngn, int scale,
                double dens_th, int64_t particle_th, const int32_t* pslot, const unsigned long long* mtot,
                int32_t* halo_id, cwthf_ms_halo* cat, int64_t cat_cap, int64_t* n_halo, cudaStream_t s) {
    const int64_t slot_cap = int64_t(ng) * ng * ng / 8 + 8;
    const int blocks = ctx->sm_count * 8;
    const int pblocks = int(std::min<int64_t>(div_up(std::max<int64_t>(np, 1), kThreads), int64_t(ctx->sm_count) * 16));
    FilterArgs f;
    f.ng = ng;
    f.L = L;
    f.mass_unit = mass_unit;
    f.dens_th = dens_th;
    f.particle_th = particle_th;
    f.cat_cap = cat_cap;
    CWTHF_LAUNCH(ctx, s, "k_ms_keep", k_ms_keep<<<blocks, kThreads, 0, s>>>(ctx->acc, ctx->seed_list, ctx->n_seeds, mtot, f,
                                                                           C, Cn, ngn, ctx->keep_off));
    int rc = scan_u32_dev(ctx, ctx->keep_off, ctx->keep_off, ctx->n_seeds, slot_cap, s);
    if (rc) return rc;
    const uint32_t* keep = ctx->keep_off;  // ranks of the halos of this scale
    const int32_t* bound = nullptr;
    if (vel) {
        // step 9: the self-boundness check of the kept groups' candidates
        CWTHF_LAUNCH(ctx, s, "k_ms_ub_group",
                     k_ms_ub_group<<<pblocks, kThreads, 0, s>>>(pslot, halo_id, np, ctx->keep_off, ctx->ub_grp));
        CWTHF_LAUNCH(ctx, s, "k_ms_ub_count",
                     k_ms_ub_count<<<1, 1, 0, s>>>(ctx->keep_off, ctx->n_seeds, ctx->ub_ngroups));
        if ((rc = unbind_groups(ctx, pos, vel, mass, mass_unit, np, L, G, ctx->ub_grp, slot_cap, ctx->ub_ngroups,
                                max_iter, ctx->ub_out, ctx->ub_nk, ctx->ub_it, s)))
            return rc;
        CWTHF_LAUNCH(ctx, s, "k_ms_ub_keep",
                     k_ms_ub_keep<<<blocks, kThreads, 0, s>>>(ctx->n_seeds, ctx->keep_off, ctx->ub_nk, ctx->acc,
                                                              ctx->ub_keep));
        if ((rc = scan_u32_dev(ctx, ctx->ub_keep, ctx->ub_keep, ctx->n_seeds, slot_cap, s))) return rc;
        const DepArgs a = make_dep_args(pos, mass, mass_unit, np, L, ng);
        CWTHF_LAUNCH(ctx, s, "k_ms_ub_sums",
                     k_ms_ub_sums<<<pblocks, kThreads, 0, s>>>(a, pslot, ctx->ub_out, ctx->seed_list, ctx->acc));
        keep = ctx->ub_keep;
        bound = ctx->ub_out;
    }
    CWTHF_LAUNCH(ctx, s, "k_ms_catalogue",
                 k_ms_catalogue<<<blocks, kThreads, 0, s>>>(ctx->acc, ctx->seed_list, ctx->n_seeds, keep, f, C,
                                                            Cn, ngn, scale, n_halo, cat, ctx->slot_halo));
    CWTHF_LAUNCH(ctx, s, "k_ms_ids", k_ms_ids<<<pblocks, kThreads, 0, s>>>(pslot, np, ctx->slot_halo, bound, halo_id));
    CWTHF_LAUNCH(ctx, s, "k_ms_advance", k_ms_advance<<<1, 1, 0, s>>>(keep, ctx->n_seeds, n_halo, cat_cap,
                                                                     ctx->d_status));
    return cuda_status(cudaGetLastError());
}

int assign_impl(cwthf_ctx* ctx, const float* pos, const float* mass, double mass_unit, int64_t np, double L, int ng,
                const int32_t* label, const float* cwt, const cwthf_params* p, int scale, int n_scales,
                int32_t* halo_id, cwthf_halo* cat, int64_t cat_cap, int64_t* n_halo, bool seeds_ready,
                bool bins_ready, cudaStream_t s) {
    int rc;
    if (!seeds_ready && (rc = seeds_from_labels(ctx, label, ng, s))) return rc;
    if (!bins_ready && (rc = bin_particles(ctx, pos, mass, mass_unit, np, L, ng, s))) return rc;
    int64_t cells = int64_t(ng) * ng * ng;
    const uint32_t* d_nseeds = ctx->n_seeds;  // seeds in use (clamped to slot_cap)
    int64_t slot_cap = cells / 8 + 8;
    int blocks = ctx->sm_count * 8;
    cudaError_t e = cudaMemsetAsync(ctx->d_mtot, 0, 8, s);
    if (e != cudaSuccess) return cuda_status(e);
    if (!seeds_ready)  // after segment_impl the resolve pass has counted the cells already
        CWTHF_LAUNCH(ctx, s, "k_count_cells",
                     k_count_cells<<<blocks, kThreads, 0, s>>>(label, cells, ctx->seed_bits, ctx->seed_prefix,
                                                               d_nseeds, ctx->acc, ctx->d_status));
    DepArgs a = make_dep_args(pos, mass, mass_unit, np, L, ng);
    const int64_t total_key = deposit_geom(ng).ntiles * kDepClasses;  // dep_off[total_key] = records binned
    int pblocks = int(std::min<int64_t>(div_up(std::max<int64_t>(np, 1), kThreads), int64_t(ctx->sm_count) * 16));
    launch_halo_sums(ctx, s, np, a, ctx->dep_off + total_key, ctx->dep_rec, ctx->dep_mq, label, ctx->seed_bits,
                     ctx->seed_prefix, d_nseeds, ctx->acc, ctx->part_slot + int64_t(scale) * np, 1, ctx->d_mtot, 0);
    FilterArgs f;
    f.ng = ng;
    f.L = L;
    f.mass_unit = mass_unit;
    f.dens_th = p->dens_th;
    f.particle_th = p->particle_th;
    f.cat_cap = cat_cap;
    CWTHF_LAUNCH(ctx, s, "k_keep", k_keep<<<blocks, kThreads, 0, s>>>(ctx->acc, d_nseeds, ctx->d_mtot, f, ctx->keep_off));
    if ((rc = scan_u32_dev(ctx, ctx->keep_off, ctx->keep_off, d_nseeds, slot_cap, s))) return rc;
    CWTHF_LAUNCH(ctx, s, "k_catalogue",
                 k_catalogue<<<blocks, kThreads, 0, s>>>(ctx->acc, ctx->seed_list, d_nseeds, ctx->keep_off, cwt, f,
                                                         cat, ctx->slot_halo + int64_t(scale) * slot_cap, n_halo,
                                                         ctx->d_status));
    if (scale == n_scales - 1) {  // halo ids of all scales at once
        const int rs = slot_group_stride(n_scales);
        const uint32_t* total = ctx->dep_off + total_key;
        if (rs == 1) launch_ids<1>(ctx, s, blocks, pblocks, np, total, n_scales, slot_cap, halo_id);
        else if (rs == 2) launch_ids<2>(ctx, s, blocks, pblocks, np, total, n_scales, slot_cap, halo_id);
        else launch_ids<4>(ctx, s, blocks, pblocks, np, total, n_scales, slot_cap, halo_id);
    }
    return cuda_status(cudaGetLastError());
}

}  // namespace cwthf
