// deposit.cu -- cloud-in-cell deposit (Sec. 2.1, Eq. 1) as exact int64 fixed
// point, binned by grid tile so that each tile is accumulated once in shared
// memory and written with plain coalesced stores (no global atomics on the
// grid, no memset of the grid).
//
// Particle i with fixed-point coordinate q = n*2^10 + f per axis gives node n
// the weight 2^10 - f and node n+1 (periodic) the weight f; the product of the
// three axis weights times the integer mass m_q is added to each of the 8
// nodes.  Integer sums are exact and independent of order, so the grid is
// bit-for-bit deterministic.
//
// Binning: a particle belongs to the tile holding its base node (n_x, n_y,
// n_z).  Its boundary class has bit a set when the node n+1 along axis a lies
// in another tile (or wraps around the box).  The tile kernel reads its own
// bin plus, from each of its 7 lower neighbours, the classes whose bits cover
// that neighbour's offset: exactly the particles that reach into the tile.
#include "internal.cuh"
#include "quant.cuh"

namespace cwthf {
namespace {

constexpr int kCountThreads = 256;
// Four warps per tile CTA: a tile's phases are separated by barriers, so
// several mid-sized CTAs per SM keep more tiles in flight than a few large
// ones (two warps per CTA measured slower: too few threads for the write-out).
constexpr int kTileThreads = 128;
constexpr int kTileCtasPerSm = 10;
constexpr unsigned kFull = 0xffffffffu;
constexpr uint32_t kInvalidKey = 0xffffffffu;
using u64 = unsigned long long;

struct PartBin {
    uint32_t key;  // tile * 8 + class, or kInvalidKey
    unsigned long long rec;
    uint32_t mq;
    int status;
};

__device__ __forceinline__ PartBin bin_particle(const DepArgs& a, int64_t i) {
    PartBin b;
    b.key = kInvalidKey;
    b.rec = 0;
    b.mq = 0;
    b.status = CWTHF_OK;
    int64_t q[3];
    const float* p = a.pos + 3 * i;
    bool ok = quantise(p[0], a.scale_m, a.scale_e, a.modulus, q[0]) && quantise(p[1], a.scale_m, a.scale_e, a.modulus, q[1]) &&
              quantise(p[2], a.scale_m, a.scale_e, a.modulus, q[2]);
    if (!ok) { b.status = CWTHF_E_BAD_INPUT; return b; }
    int ms = mass_quantum(a, i, b.mq);
    if (ms != CWTHF_OK) { b.status = ms; b.mq = 0; return b; }
    const int T[3] = {kDepTX, kDepTY, kDepTZ};
    int n[3], t[3], cls = 0;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        n[d] = int(q[d] >> kFracBits);
        t[d] = n[d] / T[d];
        if (n[d] + 1 == a.ng || (n[d] + 1) % T[d] == 0) cls |= 1 << d;
    }
    uint32_t tile = uint32_t((int64_t(t[2]) * a.nty + t[1]) * a.ntx + t[0]);
    b.key = tile * kDepClasses + uint32_t(cls);
    b.rec = pack_rec(q[0], q[1], q[2]);
    return b;
}

// Pass 1: particles per (tile, class) and the integer mass total.
__global__ void __launch_bounds__(kCountThreads) k_dep_count(DepArgs a, uint32_t* __restrict__ count,
                                                            unsigned long long* __restrict__ mtot, int* status) {
    int lane = threadIdx.x & 31;
    int64_t stride = int64_t(gridDim.x) * blockDim.x;
    unsigned long long msum = 0;
    for (int64_t base = int64_t(blockIdx.x) * blockDim.x + (threadIdx.x & ~31); base < a.np; base += stride) {
        int64_t i = base + lane;  // base is warp-uniform: every lane runs every iteration
        PartBin b;
        b.key = kInvalidKey;
        b.mq = 0;
        b.status = CWTHF_OK;
        if (i < a.np) b = bin_particle(a, i);
        if (b.status != CWTHF_OK) set_status(status, b.status);
        msum += b.mq;
        unsigned peers = __match_any_sync(kFull, b.key);
        if (b.key != kInvalidKey && lane == __ffs(peers) - 1) atomicAdd(&count[b.key], uint32_t(__popc(peers)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) msum += __shfl_xor_sync(kFull, msum, o);
    if (lane == 0 && msum) atomicAdd(mtot, msum);
}

// Pass 2: write each particle's packed record into its (tile, class) segment,
// and (when part_rec is given) the record's position in particle order
// (0xffffffff for a particle that was not binned).
__global__ void __launch_bounds__(kCountThreads) k_dep_scatter(DepArgs a, uint32_t* __restrict__ cursor,
                                                              unsigned long long* __restrict__ rec,
                                                              uint32_t* __restrict__ rec_mq,
                                                              uint32_t* __restrict__ part_rec, int* status) {
    int lane = threadIdx.x & 31;
    int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t base = int64_t(blockIdx.x) * blockDim.x + (threadIdx.x & ~31); base < a.np; base += stride) {
        int64_t i = base + lane;
        PartBin b;
        b.key = kInvalidKey;
        b.status = CWTHF_OK;
        if (i < a.np) b = bin_particle(a, i);
        unsigned peers = __match_any_sync(kFull, b.key);
        int leader = __ffs(peers) - 1;
        uint32_t slot = 0;
        if (b.key != kInvalidKey && lane == leader) slot = atomicAdd(&cursor[b.key], uint32_t(__popc(peers)));
        slot = __shfl_sync(kFull, slot, leader);
        if (b.key != kInvalidKey) {
            slot += __popc(peers & ((1u << lane) - 1));
            if (index_ok(slot, a.np, status)) {
                rec[slot] = b.rec;
                if (a.mass) rec_mq[slot] = b.mq;
            }
        }
        if (part_rec && i < a.np) part_rec[i] = b.key != kInvalidKey ? slot : 0xffffffffu;
    }
}

// The 27 (neighbour offset mask m, boundary class) pairs whose particles reach
// into a tile: a particle of the lower neighbour at offset m reaches in iff
// its class has every bit of m set.
constexpr int kReachSegments = 27;

// The j-th (neighbour offset mask m, boundary class) pair in (m, class) order.
__device__ __forceinline__ void reach_pair(int j, int& m, int& cls) {
    int n = 0;
    m = 0;
    cls = 0;
    for (int mm = 0; mm < 8; mm++)
        for (int cc = 0; cc < 8; cc++)
            if ((cc & mm) == mm) {
                if (n == j) { m = mm; cls = cc; }
                n++;
            }
}

// Pass 3: one tile at a time per CTA.  Warp 0 fetches the record ranges of
// the 27 reaching-in segments (those of the next tile while the current one is
// written out) and scans them with shuffles; the CTA processes them as one
// flattened list, so every warp works on full batches whatever the segment
// sizes; the write-out also clears the shared accumulators for the next tile.
// Three barriers per tile.
//
// Dense tiles (a clump's core can put millions of records into one tile) are
// split when a part list is given: the tile pass (kParts false) takes a
// tile's first kTileSplit records and stores the tile as usual, and lists the
// remaining parts of kTileSplit records; the part pass (kParts true, launched
// after it) spreads those parts over all CTAs, each accumulating its part in
// shared memory and adding the nonzero cells to the grid with 64-bit atomics.
// Integer sums do not depend on their order, so the grid is the same.

struct TileParts {
    uint2* list;      // (tile, part >= 1), or nullptr: every tile whole
    uint32_t* count;  // parts listed
    uint32_t cap;
};

template <bool kParts>
__global__ void __launch_bounds__(kTileThreads, kTileCtasPerSm) k_dep_tile(DepArgs a, const uint32_t* __restrict__ off,
                                                          const unsigned long long* __restrict__ rec,
                                                          const uint32_t* __restrict__ rec_mq,
                                                          const unsigned long long* __restrict__ mtot,
                                                          int64_t* __restrict__ grid, int* status, TileParts tp) {
    constexpr int kCells = kDepTX * kDepTY * kDepTZ;
    __shared__ __align__(16) uint32_t acc_lo[kCells];
    __shared__ __align__(16) uint32_t acc_hi[kCells];
    __shared__ uint32_t seg_beg[kReachSegments], seg_pre[kReachSegments + 1];
    __shared__ uint8_t seg_m[kReachSegments];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (!kParts && blockIdx.x == 0 && threadIdx.x == 0 && *mtot >= (1ull << 33)) set_status(status, CWTHF_E_OVERFLOW);
    const int64_t ntiles = int64_t(a.ntx) * a.nty * a.ntz;
    // work items: tiles, or the listed parts
    const int64_t nitems = kParts ? int64_t(min(*tp.count, tp.cap)) : ntiles;
    auto item_tile = [&](int64_t j) -> int64_t { return kParts ? int64_t(tp.list[j].x) : j; };
    const int64_t ng = a.ng;
    const bool vec = (reinterpret_cast<uintptr_t>(grid) & 15u) == 0 && (ng & 1) == 0;  // 16-byte cell pairs
    for (int c = threadIdx.x; c < kCells; c += kTileThreads) {
        acc_lo[c] = 0u;
        acc_hi[c] = 0u;
    }
    // this lane's (m, class) pair, fixed for all tiles
    int my_m = 0, my_cls = 0;
    if (warp == 0 && lane < kReachSegments) reach_pair(lane, my_m, my_cls);
    // record range of this lane's segment of tile t (warp 0 only)
    auto fetch = [&](int64_t t, uint32_t& b, uint32_t& e) {
        b = e = 0;
        if (t < ntiles && lane < kReachSegments) {
            const int tx = int(t % a.ntx), ty = int((t / a.ntx) % a.nty), tz = int(t / (int64_t(a.ntx) * a.nty));
            const int sx = tx - (my_m & 1) < 0 ? a.ntx - 1 : tx - (my_m & 1);
            const int sy = ty - ((my_m >> 1) & 1) < 0 ? a.nty - 1 : ty - ((my_m >> 1) & 1);
            const int sz = tz - ((my_m >> 2) & 1) < 0 ? a.ntz - 1 : tz - ((my_m >> 2) & 1);
            const int64_t key = ((int64_t(sz) * a.nty + sy) * a.ntx + sx) * kDepClasses + my_cls;
            b = off[key];
            e = off[key + 1];
        }
    };
    uint32_t nb = 0, ne = 0;
    if (warp == 0) fetch(blockIdx.x < nitems ? item_tile(blockIdx.x) : ntiles, nb, ne);
    for (int64_t j = blockIdx.x; j < nitems; j += gridDim.x) {
        const int64_t t = item_tile(j);  // a listed tile out of range fetches no records and writes nothing
        if (kParts && threadIdx.x == 0) (void)index_ok(t, ntiles, status);
        const int tx = int(t % a.ntx), ty = int((t / a.ntx) % a.nty), tz = int(t / (int64_t(a.ntx) * a.nty));
        const int x0 = tx * kDepTX, y0 = ty * kDepTY, z0 = tz * kDepTZ;
        const int wx = min(kDepTX, a.ng - x0), wy = min(kDepTY, a.ng - y0), wz = min(kDepTZ, a.ng - z0);
        if (warp == 0) {
            // inclusive scan of the 27 segment sizes
            uint32_t n = ne - nb, incl = n;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += y;
            }
            if (lane < kReachSegments) {
                seg_beg[lane] = nb;
                seg_pre[lane + 1] = incl;
                seg_m[lane] = uint8_t(my_m);
            }
            if (lane == 0) seg_pre[0] = 0;
        }
        __syncthreads();
        const uint32_t total = seg_pre[kReachSegments];
        // this pass's records of the tile's flattened list
        uint32_t kbeg = 0, kend = total;
        if (kParts) {
            kbeg = tp.list[j].y * kTileSplit;
            kend = min(total, kbeg + kTileSplit);
        } else if (tp.list && total > kTileSplit) {
            kend = kTileSplit;
            if (threadIdx.x == 0) {
                const uint32_t extra = (total - 1) / kTileSplit;  // parts after the first
                const uint32_t p0 = atomicAdd(tp.count, extra);
                if (p0 + extra > tp.cap) set_status(status, CWTHF_E_OVERFLOW);  // cannot happen: the list holds 8 np / split
                for (uint32_t p = 0; p < extra && p0 + p < tp.cap; p++) tp.list[p0 + p] = make_uint2(uint32_t(t), p + 1);
            }
        }
        for (uint32_t k0 = kbeg + (threadIdx.x & ~31u); k0 < kend; k0 += kTileThreads) {  // warp-uniform trip count
            const uint32_t k = k0 + uint32_t(lane);
            int sgi = 0;  // segment of k: last j with seg_pre[j] <= k
#pragma unroll
            for (int w = 16; w > 0; w >>= 1)
                if (sgi + w < kReachSegments && seg_pre[sgi + w] <= k) sgi += w;
            const uint32_t r = seg_beg[sgi] + (k - seg_pre[sgi]);
            const int m = seg_m[sgi];
            const bool live = k < kend && index_ok(r, a.np, status);
            const u64 e = live ? rec[r] : 0ull;
            const uint32_t mq = live ? (a.mass ? rec_mq[r] : 1u) : 0u;
            const int qx = rec_q(e, 0), qy = rec_q(e, 1), qz = rec_q(e, 2);
            int lx = (qx >> kFracBits) - x0, ly = (qy >> kFracBits) - y0, lz = (qz >> kFracBits) - z0;
            const int fx = qx & (kFracOne - 1), fy = qy & (kFracOne - 1), fz = qz & (kFracOne - 1);
            // a particle of a lower neighbour only reaches in with its upper node
            if (m & 1) lx = -1;
            if (m & 2) ly = -1;
            if (m & 4) lz = -1;
            // corner weights: products of three factors <= 2^kFracBits fit 32 bits
            static_assert(3 * kFracBits <= 32, "corner weight product");
            const uint32_t wxv[2] = {uint32_t(kFracOne - fx), uint32_t(fx)};
            const uint32_t wyv[2] = {uint32_t(kFracOne - fy), uint32_t(fy)};
            const uint32_t wzv[2] = {uint32_t(kFracOne - fz), uint32_t(fz)};
            // a warp whose 32 records all share one base cell (dense clumps) folds its
            // 8 corner sums with full-warp reductions; otherwise every lane adds its own
            // corners (native 32-bit shared atomics; same-cell lanes serialise briefly)
            const uint32_t key = live ? uint32_t(((lz + 1) * (kDepTY + 2) + (ly + 1)) * (kDepTX + 2) + (lx + 1))
                                      : kInvalidKey;
            const bool uniform = __all_sync(kFull, key == __shfl_sync(kFull, key, 0)) && key != kInvalidKey;
#pragma unroll
            for (int q = 0; q < 8; q++) {
                const int ex = q & 1, ey = (q >> 1) & 1, ez = (q >> 2) & 1;
                u64 v = u64(mq) * (wxv[ex] * wyv[ey] * wzv[ez]);
                if (uniform) v = warp_sum64(v);  // warp-uniform branch
                const int cx = lx + ex, cy = ly + ey, cz = lz + ez;
                if (live && (!uniform || lane == 0) && v && cx >= 0 && cx < wx && cy >= 0 && cy < wy && cz >= 0 &&
                    cz < wz)
                    shared_add64(acc_lo, acc_hi, (cz * kDepTY + cy) * kDepTX + cx, v);
            }
        }
        __syncthreads();
        if (warp == 0)  // the next item's ranges, in flight during the write-out
            fetch(j + gridDim.x < nitems ? item_tile(j + gridDim.x) : ntiles, nb, ne);
        if (kParts) {
            // a part: its nonzero cells are added to the grid
            for (int c = threadIdx.x; c < kCells; c += kTileThreads) {
                const int cx = c % kDepTX, cy = (c / kDepTX) % kDepTY, cz = c / (kDepTX * kDepTY);
                const u64 v = (u64(acc_hi[c]) << 32) | u64(acc_lo[c]);
                if (v && cx < wx && cy < wy && cz < wz)
                    atomicAdd(reinterpret_cast<u64*>(grid + (int64_t(z0 + cz) * ng + (y0 + cy)) * ng + (x0 + cx)), v);
                acc_lo[c] = 0u;
                acc_hi[c] = 0u;
            }
        } else if (vec && wx == kDepTX && wy == kDepTY && wz == kDepTZ) {
            // a whole tile: two cells per thread and step, one 16-byte store each
            // (a warp writes two 256-byte row segments)
            int64_t* tg = grid + (int64_t(z0) * ng + y0) * ng + x0;
            const int32_t plane = int32_t(ng) * int32_t(ng);
            for (int c = 2 * threadIdx.x; c < kCells; c += 2 * kTileThreads) {
                const int cx = c & (kDepTX - 1), cy = (c / kDepTX) & (kDepTY - 1), cz = c / (kDepTX * kDepTY);
                const uint2 lo = *reinterpret_cast<const uint2*>(&acc_lo[c]);
                const uint2 hi = *reinterpret_cast<const uint2*>(&acc_hi[c]);
                *reinterpret_cast<uint4*>(tg + (cz * plane + cy * int32_t(ng) + cx)) = make_uint4(lo.x, hi.x, lo.y, hi.y);
                *reinterpret_cast<uint2*>(&acc_lo[c]) = make_uint2(0u, 0u);
                *reinterpret_cast<uint2*>(&acc_hi[c]) = make_uint2(0u, 0u);
            }
        } else {
            for (int c = threadIdx.x; c < kCells; c += kTileThreads) {
                const int cx = c % kDepTX, cy = (c / kDepTX) % kDepTY, cz = c / (kDepTX * kDepTY);
                if (cx < wx && cy < wy && cz < wz)
                    grid[(int64_t(z0 + cz) * ng + (y0 + cy)) * ng + (x0 + cx)] =
                        int64_t((u64(acc_hi[c]) << 32) | u64(acc_lo[c]));
                acc_lo[c] = 0u;
                acc_hi[c] = 0u;
            }
        }
        __syncthreads();
    }
}

}  // namespace

int bin_particles(cwthf_ctx* ctx, const float* pos, const float* mass, double mass_unit, int64_t np, double L, int ng,
                  cudaStream_t s) {
    DepositGeom g = deposit_geom(ng);
    DepArgs a = make_dep_args(pos, mass, mass_unit, np, L, ng);
    int64_t nkeys = g.ntiles * kDepClasses;
    cudaError_t e;
    if ((e = cudaMemsetAsync(ctx->dep_count, 0, size_t(nkeys) * 4, s)) != cudaSuccess) return cuda_status(e);
    if ((e = cudaMemsetAsync(ctx->d_mtot, 0, 8, s)) != cudaSuccess) return cuda_status(e);
    int blocks = int(std::min<int64_t>(div_up(std::max<int64_t>(np, 1), kCountThreads), int64_t(ctx->sm_count) * 16));
    CWTHF_LAUNCH(ctx, s, "k_dep_count", k_dep_count<<<blocks, kCountThreads, 0, s>>>(a, ctx->dep_count, ctx->d_mtot, ctx->d_status));
    int rc = scan_u32(ctx, ctx->dep_count, ctx->dep_off, nkeys, s);
    if (rc) return rc;
    if ((e = cudaMemcpyAsync(ctx->dep_cursor, ctx->dep_off, size_t(nkeys) * 4, cudaMemcpyDeviceToDevice, s)) !=
        cudaSuccess)
        return cuda_status(e);
    CWTHF_LAUNCH(ctx, s, "k_dep_scatter", k_dep_scatter<<<blocks, kCountThreads, 0, s>>>(a, ctx->dep_cursor, ctx->dep_rec, ctx->dep_mq,
                                                                        ctx->part_rec, ctx->d_status));
    return cuda_status(cudaGetLastError());
}

int deposit_impl(cwthf_ctx* ctx, const float* pos, const float* mass, double mass_unit, int64_t np, double L,
                 int ng, int64_t* grid, int64_t* mtot, cudaStream_t s) {
    int rc = bin_particles(ctx, pos, mass, mass_unit, np, L, ng, s);
    if (rc) return rc;
    DepositGeom g = deposit_geom(ng);
    DepArgs a = make_dep_args(pos, mass, mass_unit, np, L, ng);
    int tblocks = int(std::min<int64_t>(g.ntiles, int64_t(ctx->sm_count) * kTileCtasPerSm));
    cudaError_t e;
    TileParts tp;
    tp.list = reinterpret_cast<uint2*>(ctx->dep_parts);
    tp.count = ctx->dep_nparts;
    tp.cap = uint32_t(tile_parts_cap(ctx->max_np));
    if ((e = cudaMemsetAsync(tp.count, 0, 4, s)) != cudaSuccess) return cuda_status(e);
    CWTHF_LAUNCH(ctx, s, "k_dep_tile", k_dep_tile<false><<<tblocks, kTileThreads, 0, s>>>(a, ctx->dep_off, ctx->dep_rec, ctx->dep_mq, ctx->d_mtot, grid,
                                                ctx->d_status, tp));
    // the dense tiles' further parts (returns at once when there are none)
    CWTHF_LAUNCH(ctx, s, "k_dep_parts",
                 k_dep_tile<true><<<ctx->sm_count * kTileCtasPerSm, kTileThreads, 0, s>>>(
                     a, ctx->dep_off, ctx->dep_rec, ctx->dep_mq, ctx->d_mtot, grid, ctx->d_status, tp));
    if (mtot && (e = cudaMemcpyAsync(mtot, ctx->d_mtot, 8, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
        return cuda_status(e);
    return cuda_status(cudaGetLastError());
}

// The same three passes on caller-provided scratch instead of a context's
// (no allocation, no context; used by the fixed-scratch entry point).
int deposit_into_scratch(const DepositScratch& sc, const float* pos, const float* mass, double mass_unit, int64_t np,
                         double L, int ng, int64_t* grid, cudaStream_t s) {
    DepositGeom g = deposit_geom(ng);
    DepArgs a = make_dep_args(pos, mass, mass_unit, np, L, ng);
    int64_t nkeys = g.ntiles * kDepClasses;
    cudaError_t e;
    if ((e = cudaMemsetAsync(sc.count, 0, size_t(nkeys) * 4, s)) != cudaSuccess) return cuda_status(e);
    if ((e = cudaMemsetAsync(sc.mtot, 0, 8, s)) != cudaSuccess) return cuda_status(e);
    int blocks = int(std::min<int64_t>(div_up(std::max<int64_t>(np, 1), kCountThreads), int64_t(sc.sm_count) * 16));
    k_dep_count<<<blocks, kCountThreads, 0, s>>>(a, sc.count, sc.mtot, sc.status);
    int rc = scan_u32_scratch(sc.count, sc.off, nkeys, sc.scan_tmp, sc.scan_cap, s);
    if (rc) return rc;
    if ((e = cudaMemcpyAsync(sc.cursor, sc.off, size_t(nkeys) * 4, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
        return cuda_status(e);
    k_dep_scatter<<<blocks, kCountThreads, 0, s>>>(a, sc.cursor, sc.rec, sc.mq, nullptr, sc.status);
    int tblocks = int(std::min<int64_t>(g.ntiles, int64_t(sc.sm_count) * kTileCtasPerSm));
    TileParts whole;  // no part list: every tile whole
    whole.list = nullptr;
    whole.count = nullptr;
    whole.cap = 0;
    k_dep_tile<false><<<tblocks, kTileThreads, 0, s>>>(a, sc.off, sc.rec, sc.mq, sc.mtot, grid, sc.status, whole);
    return cuda_status(cudaGetLastError());
}

}  // namespace cwthf
