// unbind.cu -- the self-boundness check (Sec. 2.3; step 9 of the Sec. 2 step
// list), one CTA per group, or the whole grid for a large group.
//
// For every group g, following Sec. 2.3 in order:
//   1. the centre is the centre of mass of the current members (mass-weighted
//      minimum-image offsets from the group's first member in particle order);
//   2. with spherical symmetry the potential at member i is that of the
//      shells of the other members about the centre (shell theorem):
//      Phi_i = -G sum_{j != i} m_j / max(r_i, r_j), escape speed^2 = -2 Phi_i;
//      with the members sorted by radius this is
//      Phi_i = -G (M(before i) / r_i + sum_{j after i} m_j / r_j);
//   3. members faster than their escape speed, relative to the group's
//      mass-weighted mean velocity, are excluded, all at once;
//   4. steps 1-3 repeat until nothing is excluded (at most max_iter rounds);
//   5. a group that lost more than 40 % of its particles is discarded.
// Each round: fixed-order block reductions (the sums do not depend on timing),
// a sort of the radii (bitonic in shared memory for small groups, a stable
// radix sort in the group's slice of global scratch for larger ones), chunked
// block scans for the shell sums, and a stable compaction of the members that
// stay.  Groups above a size threshold are processed by the whole grid instead
// (k_ub_grid, one group at a time), with the same steps over per-CTA chunks.
#include <algorithm>
#include <cmath>

#include "internal.cuh"

namespace cwthf {
namespace {

constexpr int kUbThreads = 512;
constexpr int kUbWarps = kUbThreads / 32;
constexpr int kUbSmemElems = 2048;  // groups up to this size sort in shared memory

// Integer mass quanta (the deposit's rule): 1 when masses are equal, else
// rint(m / mass_unit); invalid masses are reported once here.
__global__ void k_ub_count(const float* __restrict__ mass, double mass_unit, const int32_t* __restrict__ group,
                           int64_t np, int64_t n_groups, const uint32_t* __restrict__ d_groups,
                           uint32_t* __restrict__ cnt, int32_t* __restrict__ group_out, int* status) {
    if (d_groups) n_groups = *d_groups;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < np; i += stride) {
        group_out[i] = -1;
        if (mass) {
            const double r = rint(__ddiv_rn(double(mass[i]), mass_unit));
            if (!(r >= 0.0)) set_status(status, CWTHF_E_BAD_INPUT);
            else if (!(r < 2147483648.0)) set_status(status, CWTHF_E_OVERFLOW);
        }
        const int32_t g = group[i];
        if (g >= 0 && int64_t(g) < n_groups) atomicAdd(&cnt[g], 1u);
    }
}

__global__ void k_ub_scatter(const int32_t* __restrict__ group, int64_t np, int64_t n_groups,
                             const uint32_t* __restrict__ d_groups, const uint32_t* __restrict__ off,
                             uint32_t* __restrict__ cur, int32_t* __restrict__ mem, int* status) {
    if (d_groups) n_groups = *d_groups;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < np; i += stride) {
        const int32_t g = group[i];
        if (g >= 0 && int64_t(g) < n_groups) {
            const uint32_t k = off[g] + atomicAdd(&cur[g], 1u);
            if (index_ok(k, np, status)) mem[k] = int32_t(i);
        }
    }
}

struct UbArgs {
    const float* pos;
    const float* vel;
    const float* mass;
    double mass_unit, L, G;
    const uint32_t* off;  // [n_groups + 1] first member of each group in mem
    int32_t* mem;         // [np] members, grouped
    uint64_t* key;        // [2 np] sort keys (group g of n members: 2 n entries from 2 off[g], the
                          // pairs and the radix sort's other buffer)
    int32_t* val;         // [2 np] sort values (the same layout)
    int max_iter;
    int64_t grid_min;            // larger groups are left to the whole-grid path
    int64_t n_groups;            // groups (or read from d_groups when given)
    const uint32_t* d_groups;
    int32_t* group_out;
    int64_t* n_kept;
    int32_t* iters;
};

__device__ __forceinline__ double mass_of(const UbArgs& a, int32_t i) {
    const double q = a.mass ? rint(__ddiv_rn(double(a.mass[i]), a.mass_unit)) : 1.0;
    return __dmul_rn(q, a.mass_unit);
}

// minimum-image offset of coordinate x from the anchor coordinate x0
__device__ __forceinline__ double min_image(float x, float x0, double L) {
    const double d = __dsub_rn(double(x), double(x0));
    return __dsub_rn(d, __dmul_rn(L, floor(__dadd_rn(__ddiv_rn(d, L), 0.5))));
}

// Sums of NV values over the block in a fixed order (warp trees, then one
// warp over the warp totals): the result does not depend on timing.
template <int NV>
__device__ __forceinline__ void block_sums(double (&v)[NV], double* sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; k++)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; k++) sh[k * kUbWarps + w] = v[k];
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int k = 0; k < NV; k++) {
            double x = lane < kUbWarps ? sh[k * kUbWarps + lane] : 0.0;
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
            if (lane == 0) sh[k * kUbWarps] = x;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; k++) v[k] = sh[k * kUbWarps];
    __syncthreads();
}

// Exclusive scan of one value per thread (thread order), in a fixed order;
// *total receives the sum.
template <class T>
__device__ __forceinline__ T block_exclusive(T x, T* sh, T* total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T incl = x;
    for (int o = 1; o < 32; o <<= 1) {
        const T y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) sh[w] = incl;
    __syncthreads();
    if (w == 0) {
        T s = lane < kUbWarps ? sh[lane] : T(0);
        T si = s;
        for (int o = 1; o < 32; o <<= 1) {
            const T y = __shfl_up_sync(0xffffffffu, si, o);
            if (lane >= o) si += y;
        }
        if (lane < kUbWarps) sh[lane] = si - s;  // exclusive warp offsets
        if (lane == kUbWarps - 1) sh[kUbWarps] = si;
    }
    __syncthreads();
    const T r = sh[w] + incl - x;
    *total = sh[kUbWarps];
    __syncthreads();
    return r;
}

// Bitonic sort of P (a power of two) (key, value) pairs, ascending keys.
template <class K>
__device__ void bitonic(K* k, int32_t* v, int P) {
    for (int size = 2; size <= P; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < P / 2; t += blockDim.x) {
                const int lo = (t / stride) * 2 * stride + (t % stride), hi = lo + stride;
                const bool up = (lo & size) == 0;
                const K a = k[lo], b = k[hi];
                if ((a > b) == up) {
                    k[lo] = b;
                    k[hi] = a;
                    const int32_t va = v[lo];
                    v[lo] = v[hi];
                    v[hi] = va;
                }
            }
            __syncthreads();
        }
}

// Stable LSD radix sort (8-bit digits, the lowest nbytes bytes of the keys)
// of the n pairs K[0..n), V[0..n), with K[n..2n), V[n..2n) as the other
// buffer; the result ends in K[0..n), V[0..n).  Every warp owns a contiguous
// chunk: per pass, per-warp digit counts (shared memory), their offsets
// digit-major then warp by warp, and a scatter that keeps each warp's chunk in
// order (lanes of one digit ranked by match_any).  A pass in which every key
// has the same digit moves nothing and is skipped.  All threads of the block.
__device__ void radix_sort_pairs(uint64_t* K, int32_t* V, int n, int nbytes, uint32_t* hist, int* skip) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int chunk = (n + nw - 1) / nw;
    const int c0 = min(n, warp * chunk), c1 = min(n, c0 + chunk);
    const uint32_t lt = (1u << lane) - 1u;
    uint64_t *ka = K, *kb = K + n;
    int32_t *va = V, *vb = V + n;
    for (int pass = 0; pass < nbytes; pass++) {
        const int sh = 8 * pass;
        for (int i = threadIdx.x; i < nw * 256; i += blockDim.x) hist[i] = 0u;
        if (threadIdx.x == 0) *skip = 0;
        __syncthreads();
        for (int k = c0 + lane; k < c1; k += 32) atomicAdd(&hist[warp * 256 + int((ka[k] >> sh) & 255u)], 1u);
        __syncthreads();
        // offsets: digit d's block starts after all smaller digits; within it, warp by warp
        uint32_t tot = 0;
        if (threadIdx.x < 256)
            for (int w = 0; w < nw; w++) tot += hist[w * 256 + threadIdx.x];
        if (threadIdx.x < 256 && tot == uint32_t(n)) *skip = 1;
        // exclusive scan of the 256 digit totals (threads 0..255, 8 warps)
        __shared__ uint32_t wsum[8];
        uint32_t incl = tot;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (threadIdx.x < 256 && lane == 31) wsum[warp] = incl;
        __syncthreads();
        if (threadIdx.x < 256) {
            uint32_t base = incl - tot;
            for (int w = 0; w < warp; w++) base += wsum[w];
            for (int w = 0; w < nw; w++) {
                const uint32_t c = hist[w * 256 + threadIdx.x];
                hist[w * 256 + threadIdx.x] = base;
                base += c;
            }
        }
        __syncthreads();
        if (*skip) {  // block-uniform; the barrier keeps the next pass's reset behind every read
            __syncthreads();
            continue;
        }
        uint32_t* off = hist + warp * 256;
        for (int k0 = c0; k0 < c1; k0 += 32) {
            const int k = k0 + lane;
            const bool valid = k < c1;
            const int d = valid ? int((ka[k] >> sh) & 255u) : 256;
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            if (valid) {
                const uint32_t pos = off[d] + __popc(peers & lt);
                kb[pos] = ka[k];
                vb[pos] = va[k];
            }
            __syncwarp();
            if (valid && lane == __ffs(peers) - 1) off[d] += __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        uint64_t* tk = ka;
        ka = kb;
        kb = tk;
        int32_t* tv = va;
        va = vb;
        vb = tv;
    }
    if (ka != K) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            K[i] = ka[i];
            V[i] = va[i];
        }
    }
    __syncthreads();
}

// Sorts the group's first n pairs of (K, V) (keys below 2^(8 nbytes)): a
// bitonic sort in shared memory when the padded length fits, else the radix
// sort in the group's slice of global scratch (2n entries).
__device__ void sort_pairs(uint64_t* K, int32_t* V, int n, int nbytes, uint64_t* sk, int32_t* sv, uint32_t* hist,
                           int* skip) {
    int P = 1;
    while (P < n) P <<= 1;
    if (P <= kUbSmemElems) {
        for (int t = threadIdx.x; t < P; t += blockDim.x) {
            sk[t] = t < n ? K[t] : ~0ull;
            sv[t] = t < n ? V[t] : -1;
        }
        __syncthreads();
        bitonic(sk, sv, P);
        for (int t = threadIdx.x; t < n; t += blockDim.x) {
            K[t] = sk[t];
            V[t] = sv[t];
        }
        __syncthreads();
    } else {
        radix_sort_pairs(K, V, n, nbytes, hist, skip);
    }
}

// One group (all of the CTA's threads).
__device__ void unbind_group(const UbArgs& a, int64_t g, uint64_t* sk, int32_t* sv, double* shd, int64_t* shi,
                             uint32_t* hist, int* skip) {
    const uint32_t base = a.off[g];
    const int n0 = int(a.off[g + 1] - base);
    const int tid = threadIdx.x;
    if (int64_t(n0) > a.grid_min) return;  // the whole-grid path's group
    if (n0 == 0) {
        if (tid == 0) {
            a.n_kept[g] = 0;
            a.iters[g] = 0;
        }
        return;
    }
    int32_t* X = a.mem + base;
    uint64_t* K = a.key + 2 * size_t(base);
    int32_t* V = a.val + 2 * size_t(base);
    // members in particle order, so that every sum below runs in a fixed order
    for (int t = tid; t < n0; t += blockDim.x) {
        K[t] = uint64_t(uint32_t(X[t]));
        V[t] = X[t];
    }
    __syncthreads();
    sort_pairs(K, V, n0, 4, sk, sv, hist, skip);
    for (int t = tid; t < n0; t += blockDim.x) X[t] = V[t];
    __syncthreads();
    const float* a0 = a.pos + 3 * size_t(X[0]);
    const float ax = a0[0], ay = a0[1], az = a0[2];
    const double L = a.L, twoG = 2.0 * a.G;
    int n = n0, it = 0;
    while (it < a.max_iter) {
        it++;
        // 1. centre of mass and mean velocity
        double s[7] = {0, 0, 0, 0, 0, 0, 0};
        for (int k = tid; k < n; k += blockDim.x) {
            const int32_t i = X[k];
            const double m = mass_of(a, i);
            const float* p = a.pos + 3 * size_t(i);
            const float* v = a.vel + 3 * size_t(i);
            s[0] += m;
            s[1] += m * min_image(p[0], ax, L);
            s[2] += m * min_image(p[1], ay, L);
            s[3] += m * min_image(p[2], az, L);
            s[4] += m * double(v[0]);
            s[5] += m * double(v[1]);
            s[6] += m * double(v[2]);
        }
        block_sums<7>(s, shd);
        const double M = s[0];
        const double cx = M > 0.0 ? s[1] / M : 0.0, cy = M > 0.0 ? s[2] / M : 0.0, cz = M > 0.0 ? s[3] / M : 0.0;
        const double vx = M > 0.0 ? s[4] / M : 0.0, vy = M > 0.0 ? s[5] / M : 0.0, vz = M > 0.0 ? s[6] / M : 0.0;
        // radii about the centre, sorted
        for (int t = tid; t < n; t += blockDim.x) {
            const int32_t i = X[t];
            const float* p = a.pos + 3 * size_t(i);
            const double dx = __dsub_rn(min_image(p[0], ax, L), cx);
            const double dy = __dsub_rn(min_image(p[1], ay, L), cy);
            const double dz = __dsub_rn(min_image(p[2], az, L), cz);
            const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
            K[t] = uint64_t(__double_as_longlong(__dsqrt_rn(r2)));  // r >= 0: the bits order like the values
            V[t] = i;
        }
        __syncthreads();
        sort_pairs(K, V, n, 8, sk, sv, hist, skip);
        // 2-3. shell sums per member and the exclusions.  Thread t walks the
        // chunk [t ch, (t+1) ch): mass before the chunk and m/r after it come
        // from block scans of the chunk totals.  Massive members at the centre
        // (r = 0, sorted first) enter the later members' sums through the mass
        // before them; for another member at r = 0 they make the potential
        // infinite (counted apart, so no infinity enters the scans).
        const int ch = (n + blockDim.x - 1) / blockDim.x;
        const int c0 = min(n, tid * ch), c1 = min(n, c0 + ch);
        double tm = 0.0, tq = 0.0;
        long long tz = 0;
        for (int k = c0; k < c1; k++) {
            const double r = __longlong_as_double((long long)K[k]);
            const double m = mass_of(a, V[k]);
            tm += m;
            if (m > 0.0) {
                if (r > 0.0) tq += m / r;
                else tz++;
            }
        }
        double tot_m, tot_q;
        long long tot_z;
        const double pre_m = block_exclusive(tm, shd, &tot_m);
        const double pre_q = block_exclusive(tq, shd, &tot_q);
        (void)block_exclusive(tz, reinterpret_cast<long long*>(shi), &tot_z);
        const double after_q = tot_q - pre_q - tq;  // m/r of the chunks after this one
        double run_m = pre_m, run_q = 0.0;
        int nk = 0;
        for (int k = c0; k < c1; k++) {
            const int32_t i = V[k];
            const double r = __longlong_as_double((long long)K[k]);
            const double m = mass_of(a, i);
            if (m > 0.0 && r > 0.0) run_q += m / r;
            const double below = run_m > 0.0 ? run_m / r : 0.0;  // M(before) / r (r = 0: infinite)
            double S = below + (after_q + (tq - run_q));
            if (r == 0.0 && tot_z - (m > 0.0 ? 1 : 0) > 0) S = __longlong_as_double(0x7ff0000000000000ll);
            run_m += m;
            const float* v = a.vel + 3 * size_t(i);
            const double ux = double(v[0]) - vx, uy = double(v[1]) - vy, uz = double(v[2]) - vz;
            const double v2 = ux * ux + uy * uy + uz * uz;
            const bool stay = !(v2 > twoG * S);
            if (!stay) V[k] = ~i;  // marked for exclusion
            nk += stay;
        }
        long long n_keep;
        const long long dst0 = block_exclusive((long long)nk, reinterpret_cast<long long*>(shi), &n_keep);
        if (n_keep == n) break;
        // stable compaction of the members that stay
        long long d = dst0;
        for (int k = c0; k < c1; k++) {
            const int32_t i = V[k];
            if (i >= 0) X[d++] = i;
        }
        __syncthreads();
        n = int(n_keep);
    }
    // 5. more than 40 % excluded: the group is discarded
    const bool discard = 5ll * (n0 - n) > 2ll * n0;
    if (!discard)
        for (int k = tid; k < n; k += blockDim.x) a.group_out[X[k]] = int32_t(g);
    if (tid == 0) {
        a.n_kept[g] = discard ? 0 : n;
        a.iters[g] = it;
    }
}

// ---- the whole-grid path: one large group at a time, every CTA ---------------
//
// The same steps as unbind_group, with each CTA owning a contiguous chunk of
// the group's members and grid barriers between the phases.  Partial sums go
// through per-CTA slots and are combined in CTA order by every CTA, so the
// sums do not depend on timing either; the radix sort takes per-CTA digit
// counts, so its scatter keeps (CTA, warp, member) order and stays stable.
// Cross-CTA data is read with __ldcg after the barriers (L1 is not coherent).

constexpr int kUbPart = 16;  // per-CTA partial slots: 0-6 centre of mass, 8-10 shell sums, 11 kept

struct UbGrid {
    double* part;    // [gridDim][kUbPart]
    uint32_t* hist;  // [2][gridDim][256] by pass parity
    unsigned* bar;
    int* status;
};

// [b, e) of the CTA's chunk of n members
__device__ __forceinline__ void cta_chunk(int n, int& b, int& e) {
    const int ch = (n + int(gridDim.x) - 1) / int(gridDim.x);
    b = min(n, int(blockIdx.x) * ch);
    e = min(n, b + ch);
}

// Sums over the CTAs of partial slot k, in CTA order: over all CTAs (*all)
// and over the CTAs before this one (returned).  Thread-local.
__device__ __forceinline__ double part_prefix(const double* part, int k, double* all) {
    double s = 0.0, before = 0.0;
    for (int c = 0; c < int(gridDim.x); c++) {
        if (c == int(blockIdx.x)) before = s;
        s += __ldcg(part + size_t(c) * kUbPart + k);
    }
    *all = s;
    return before;
}

// The stable LSD radix sort of radix_sort_pairs over the whole grid: the
// digit offsets add the counts of all CTAs before this one.  Returns false on
// a barrier timeout.
__device__ bool grid_radix(uint64_t* K, int32_t* V, int n, int nbytes, const UbGrid& b, uint32_t* hist,
                           uint32_t* dsum, uint32_t* dbase, int* skip, int& parity) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    int C0, C1;
    cta_chunk(n, C0, C1);
    const int wch = (C1 - C0 + nw - 1) / nw;
    const int w0 = min(C1, C0 + warp * wch), w1 = min(C1, w0 + wch);
    const uint32_t lt = (1u << lane) - 1u;
    __shared__ uint32_t wsum[8];
    uint64_t *ka = K, *kb = K + n;
    int32_t *va = V, *vb = V + n;
    for (int pass = 0; pass < nbytes; pass++) {
        const int sh = 8 * pass;
        for (int i = tid; i < nw * 256; i += blockDim.x) hist[i] = 0u;
        if (tid == 0) *skip = 0;
        __syncthreads();
        for (int k = w0 + lane; k < w1; k += 32) atomicAdd(&hist[warp * 256 + int((__ldcg(ka + k) >> sh) & 255u)], 1u);
        __syncthreads();
        uint32_t* gh = b.hist + (size_t(parity) * gridDim.x + blockIdx.x) * 256;
        if (tid < 256) {
            uint32_t t = 0;
            for (int w = 0; w < nw; w++) t += hist[w * 256 + tid];
            gh[tid] = t;
        }
        if (!grid_sync(b.bar, b.status)) return false;
        if (tid < 256) {
            uint32_t all = 0, before = 0;
            const uint32_t* col = b.hist + size_t(parity) * gridDim.x * 256 + tid;
            for (int c = 0; c < int(gridDim.x); c++) {
                if (c == int(blockIdx.x)) before = all;
                all += __ldcg(col + size_t(c) * 256);
            }
            dsum[tid] = all;
            dbase[tid] = before;
            if (all == uint32_t(n)) *skip = 1;
        }
        parity ^= 1;  // the next pass writes the other copy while slower CTAs may still read this one
        __syncthreads();
        if (*skip) {  // the same decision in every CTA (same totals)
            __syncthreads();
            continue;
        }
        // digit d starts after all smaller digits of every CTA, then after the
        // CTAs before this one, then warp by warp
        const uint32_t tot = tid < 256 ? dsum[tid] : 0u;
        uint32_t incl = tot;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (tid < 256 && lane == 31) wsum[warp] = incl;
        __syncthreads();
        if (tid < 256) {
            uint32_t base = incl - tot + dbase[tid];
            for (int w = 0; w < warp; w++) base += wsum[w];
            for (int w = 0; w < nw; w++) {
                const uint32_t c = hist[w * 256 + tid];
                hist[w * 256 + tid] = base;
                base += c;
            }
        }
        __syncthreads();
        uint32_t* off = hist + warp * 256;
        for (int k0 = w0; k0 < w1; k0 += 32) {
            const int k = k0 + lane;
            const bool valid = k < w1;
            const uint64_t key = valid ? __ldcg(ka + k) : 0ull;
            const int d = valid ? int((key >> sh) & 255u) : 256;
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            if (valid) {
                const uint32_t pos = off[d] + __popc(peers & lt);
                kb[pos] = key;
                vb[pos] = __ldcg(va + k);
            }
            __syncwarp();
            if (valid && lane == __ffs(peers) - 1) off[d] += __popc(peers);
            __syncwarp();
        }
        if (!grid_sync(b.bar, b.status)) return false;  // every scatter lands before the next pass reads
        uint64_t* tk = ka;
        ka = kb;
        kb = tk;
        int32_t* tv = va;
        va = vb;
        vb = tv;
    }
    if (ka != K) {
        for (int i = C0 + tid; i < C1; i += blockDim.x) {
            K[i] = __ldcg(ka + i);
            V[i] = __ldcg(va + i);
        }
        if (!grid_sync(b.bar, b.status)) return false;
    }
    return true;
}

// One group with every CTA of the grid.  Returns false on a barrier timeout.
__device__ bool unbind_group_grid(const UbArgs& a, const UbGrid& b, int64_t g, double* shd, int64_t* shi,
                                  uint32_t* hist, uint32_t* dsum, uint32_t* dbase, int* skip, int& parity) {
    __shared__ double bc[8];
    const uint32_t base = a.off[g];
    const int n0 = int(a.off[g + 1] - base);
    const int tid = threadIdx.x;
    double* mypart = b.part + size_t(blockIdx.x) * kUbPart;
    int32_t* X = a.mem + base;
    uint64_t* K = a.key + 2 * size_t(base);
    int32_t* V = a.val + 2 * size_t(base);
    int C0, C1;
    // members in particle order
    cta_chunk(n0, C0, C1);
    for (int t = C0 + tid; t < C1; t += blockDim.x) {
        const int32_t i = X[t];
        K[t] = uint64_t(uint32_t(i));
        V[t] = i;
    }
    if (!grid_sync(b.bar, b.status)) return false;
    if (!grid_radix(K, V, n0, 4, b, hist, dsum, dbase, skip, parity)) return false;
    for (int t = C0 + tid; t < C1; t += blockDim.x) X[t] = __ldcg(V + t);
    if (!grid_sync(b.bar, b.status)) return false;
    const int32_t first = __ldcg(X);
    const float* a0 = a.pos + 3 * size_t(first);
    const float ax = a0[0], ay = a0[1], az = a0[2];
    const double L = a.L, twoG = 2.0 * a.G;
    int n = n0, it = 0;
    while (it < a.max_iter) {
        it++;
        cta_chunk(n, C0, C1);
        // 1. centre of mass and mean velocity: CTA sums, then all CTAs in order
        double s[7] = {0, 0, 0, 0, 0, 0, 0};
        for (int k = C0 + tid; k < C1; k += blockDim.x) {
            const int32_t i = __ldcg(X + k);
            const double m = mass_of(a, i);
            const float* p = a.pos + 3 * size_t(i);
            const float* v = a.vel + 3 * size_t(i);
            s[0] += m;
            s[1] += m * min_image(p[0], ax, L);
            s[2] += m * min_image(p[1], ay, L);
            s[3] += m * min_image(p[2], az, L);
            s[4] += m * double(v[0]);
            s[5] += m * double(v[1]);
            s[6] += m * double(v[2]);
        }
        block_sums<7>(s, shd);
        if (tid < 7) mypart[tid] = s[tid];
        if (!grid_sync(b.bar, b.status)) return false;
        if (tid < 7) {
            double all;
            (void)part_prefix(b.part, tid, &all);
            bc[tid] = all;
        }
        __syncthreads();
        const double M = bc[0];
        const double cx = M > 0.0 ? bc[1] / M : 0.0, cy = M > 0.0 ? bc[2] / M : 0.0, cz = M > 0.0 ? bc[3] / M : 0.0;
        const double vx = M > 0.0 ? bc[4] / M : 0.0, vy = M > 0.0 ? bc[5] / M : 0.0, vz = M > 0.0 ? bc[6] / M : 0.0;
        // radii about the centre, sorted over the grid
        for (int t = C0 + tid; t < C1; t += blockDim.x) {
            const int32_t i = __ldcg(X + t);
            const float* p = a.pos + 3 * size_t(i);
            const double dx = __dsub_rn(min_image(p[0], ax, L), cx);
            const double dy = __dsub_rn(min_image(p[1], ay, L), cy);
            const double dz = __dsub_rn(min_image(p[2], az, L), cz);
            const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
            K[t] = uint64_t(__double_as_longlong(__dsqrt_rn(r2)));
            V[t] = i;
        }
        if (!grid_sync(b.bar, b.status)) return false;
        if (!grid_radix(K, V, n, 8, b, hist, dsum, dbase, skip, parity)) return false;
        // 2-3. shell sums: thread chunks inside the CTA's chunk; the mass
        // before and m/r after come from block scans and the CTA partials
        const int ch = (C1 - C0 + int(blockDim.x) - 1) / int(blockDim.x);
        const int c0 = min(C1, C0 + tid * ch), c1 = min(C1, c0 + ch);
        double tm = 0.0, tq = 0.0;
        long long tz = 0;
        for (int k = c0; k < c1; k++) {
            const double r = __longlong_as_double((long long)__ldcg(K + k));
            const double m = mass_of(a, __ldcg(V + k));
            tm += m;
            if (m > 0.0) {
                if (r > 0.0) tq += m / r;
                else tz++;
            }
        }
        double cta_m, cta_q;
        long long cta_z;
        const double pre_m_t = block_exclusive(tm, shd, &cta_m);
        const double pre_q_t = block_exclusive(tq, shd, &cta_q);
        (void)block_exclusive(tz, reinterpret_cast<long long*>(shi), &cta_z);
        if (tid == 0) {
            mypart[8] = cta_m;
            mypart[9] = cta_q;
            mypart[10] = double(cta_z);
        }
        if (!grid_sync(b.bar, b.status)) return false;
        if (tid < 3) {
            double all;
            const double before = part_prefix(b.part, 8 + tid, &all);
            bc[tid] = before;
            bc[3 + tid] = all;
        }
        __syncthreads();
        const double pre_m = bc[0] + pre_m_t, pre_q = bc[1] + pre_q_t, tot_q = bc[4];
        const long long tot_z = (long long)bc[5];
        const double after_q = tot_q - pre_q - tq;
        double run_m = pre_m, run_q = 0.0;
        int nk = 0;
        for (int k = c0; k < c1; k++) {
            const int32_t i = __ldcg(V + k);
            const double r = __longlong_as_double((long long)__ldcg(K + k));
            const double m = mass_of(a, i);
            if (m > 0.0 && r > 0.0) run_q += m / r;
            const double below = run_m > 0.0 ? run_m / r : 0.0;
            double S = below + (after_q + (tq - run_q));
            if (r == 0.0 && tot_z - (m > 0.0 ? 1 : 0) > 0) S = __longlong_as_double(0x7ff0000000000000ll);
            run_m += m;
            const float* v = a.vel + 3 * size_t(i);
            const double ux = double(v[0]) - vx, uy = double(v[1]) - vy, uz = double(v[2]) - vz;
            const double v2 = ux * ux + uy * uy + uz * uz;
            const bool stay = !(v2 > twoG * S);
            if (!stay) V[k] = ~i;
            nk += stay;
        }
        long long cta_keep;
        const long long dst_t = block_exclusive((long long)nk, reinterpret_cast<long long*>(shi), &cta_keep);
        if (tid == 0) mypart[11] = double(cta_keep);
        if (!grid_sync(b.bar, b.status)) return false;
        if (tid == 0) {
            double all;
            const double before = part_prefix(b.part, 11, &all);
            bc[0] = before;
            bc[1] = all;
        }
        __syncthreads();
        const long long n_keep = (long long)bc[1];
        if (n_keep == n) break;  // the same in every CTA
        long long d = (long long)bc[0] + dst_t;
        for (int k = c0; k < c1; k++) {
            const int32_t i = V[k];  // this thread's own marks
            if (i >= 0) X[d++] = i;
        }
        if (!grid_sync(b.bar, b.status)) return false;
        n = int(n_keep);
    }
    const bool discard = 5ll * (n0 - n) > 2ll * n0;
    cta_chunk(n, C0, C1);
    if (!discard)
        for (int k = C0 + tid; k < C1; k += blockDim.x) a.group_out[__ldcg(X + k)] = int32_t(g);
    if (blockIdx.x == 0 && tid == 0) {
        a.n_kept[g] = discard ? 0 : n;
        a.iters[g] = it;
    }
    // the partial slots and X are reused by the next group
    return grid_sync(b.bar, b.status);
}

// The groups above a.grid_min, one after another, each with the whole grid
// (a cooperative launch: every CTA resident).  A barrier that runs out ends
// the kernel with CWTHF_E_TIMEOUT.
__global__ void __launch_bounds__(kUbThreads) k_ub_grid(UbArgs a, UbGrid b) {
    __shared__ double shd[8 * kUbWarps];
    __shared__ int64_t shi[kUbWarps + 1];
    __shared__ uint32_t hist[kUbWarps * 256];
    __shared__ uint32_t dsum[256], dbase[256];
    __shared__ int skip;
    const int64_t n_groups = a.d_groups ? int64_t(*a.d_groups) : a.n_groups;
    int parity = 0;
    for (int64_t g = 0; g < n_groups; g++) {
        if (int64_t(a.off[g + 1] - a.off[g]) <= a.grid_min) continue;
        if (!unbind_group_grid(a, b, g, shd, shi, hist, dsum, dbase, &skip, parity)) return;
    }
}

// A persistent grid over the groups: each CTA takes groups g, g + gridDim.x, ...
__global__ void __launch_bounds__(kUbThreads) k_ub_group(UbArgs a) {
    __shared__ uint64_t sk[kUbSmemElems];
    __shared__ int32_t sv[kUbSmemElems];
    __shared__ double shd[8 * kUbWarps];
    __shared__ int64_t shi[kUbWarps + 1];
    __shared__ uint32_t hist[kUbWarps * 256];
    __shared__ int skip;
    const int64_t n_groups = a.d_groups ? int64_t(*a.d_groups) : a.n_groups;
    for (int64_t g = blockIdx.x; g < n_groups; g += gridDim.x) {
        unbind_group(a, g, sk, sv, shd, shi, hist, &skip);
        __syncthreads();
    }
}

}  // namespace

int unbind_groups(cwthf_ctx* ctx, const float* pos, const float* vel, const float* mass, double mass_unit, int64_t np,
                  double L, double G, const int32_t* group, int64_t n_groups, const uint32_t* d_groups, int max_iter,
                  int32_t* group_out, int64_t* n_kept, int32_t* iters, cudaStream_t s) {
    // n_groups: the groups, or with d_groups the most there can be
    uint32_t* cnt = ctx->ub_off;
    uint32_t* cur = ctx->ub_cur;
    cudaError_t e = cudaMemsetAsync(cnt, 0, size_t(n_groups + 1) * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(cur, 0, size_t(n_groups + 1) * 4, s);
    if (e != cudaSuccess) return cuda_status(e);
    const int blocks = ctx->sm_count * 8;
    CWTHF_LAUNCH(ctx, s, "k_ub_count",
                 k_ub_count<<<blocks, 256, 0, s>>>(mass, mass_unit, group, np, n_groups, d_groups, cnt, group_out,
                                                   ctx->d_status));
    // in place: offsets, cnt[groups] = members
    int rc = d_groups ? scan_u32_dev(ctx, cnt, cnt, d_groups, n_groups, s) : scan_u32(ctx, cnt, cnt, n_groups, s);
    if (rc) return rc;
    CWTHF_LAUNCH(ctx, s, "k_ub_scatter",
                 k_ub_scatter<<<blocks, 256, 0, s>>>(group, np, n_groups, d_groups, cnt, cur, ctx->ub_mem,
                                                     ctx->d_status));
    if (n_groups > 0) {
        UbArgs a;
        a.pos = pos;
        a.vel = vel;
        a.mass = mass;
        a.mass_unit = mass_unit;
        a.L = L;
        a.G = G;
        a.off = cnt;
        a.mem = ctx->ub_mem;
        a.key = ctx->ub_key;
        a.val = ctx->ub_val;
        a.max_iter = max_iter;
        a.grid_min = ctx->dbg_unbind_grid_min;
        a.n_groups = n_groups;
        a.d_groups = d_groups;
        a.group_out = group_out;
        a.n_kept = n_kept;
        a.iters = iters;
        const unsigned grid = unsigned(std::min<int64_t>(n_groups, int64_t(ctx->sm_count) * 4));
        CWTHF_LAUNCH(ctx, s, "k_ub_group", k_ub_group<<<grid, kUbThreads, 0, s>>>(a));
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e);
        // the large groups: one cooperative launch (its barrier state starts cleared)
        if ((e = cudaMemsetAsync(ctx->ub_bar, 0, 16, s)) != cudaSuccess) return cuda_status(e);
        UbGrid b;
        b.part = ctx->ub_part;
        b.hist = ctx->ub_hist;
        b.bar = ctx->ub_bar;
        b.status = ctx->d_status;
        void* args[] = {&a, &b};
        CWTHF_LAUNCH(ctx, s, "k_ub_grid",
                     e = cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(&k_ub_grid),
                                                     dim3(unsigned(ctx->ub_grid_blocks)), dim3(kUbThreads), args, 0,
                                                     s));
        if (e != cudaSuccess) return cuda_status(e);
    }
    return cuda_status(cudaGetLastError());
}

int unbind_grid_blocks(int sm_count) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ub_grid, kUbThreads, 0) != cudaSuccess || per_sm < 1)
        return -1;
    return std::min(per_sm, 2) * sm_count;
}

int unbind_impl(cwthf_ctx* ctx, const float* pos, const float* vel, const float* mass, double mass_unit, int64_t np,
                double L, double G, const int32_t* group, int64_t n_groups, int max_iter, int32_t* group_out,
                int64_t* n_kept, int32_t* iters, cudaStream_t s) {
    return unbind_groups(ctx, pos, vel, mass, mass_unit, np, L, G, group, n_groups, nullptr, max_iter, group_out,
                         n_kept, iters, s);
}

}  // namespace cwthf
