// segment.cu -- local maxima and steepest-ascent segmentation of the CWT field
// (Sec. 2 steps 4-5, Sec. 2.3).
//
// Order on cells: a beats b iff C[a] > C[b], or C[a] == C[b] and a < b
// (a, b linear indices).  parent(c) = the best of c and its 26 periodic
// neighbours; c is a local maximum iff parent(c) == c.  A maximum with
// C > cwt_min is a seed; the label of a cell is the seed its parent chain
// reaches, or -1 when the chain ends at a maximum that is not a seed.
//
// k_seg_tile stages one tile plus a one-cell halo of C in shared memory,
// computes the parents of the tile's cells, and resolves every chain that
// stays inside the tile by pointer jumping in shared memory.  A chain that
// leaves the tile is written as a flagged pointer (bit 30) to the first cell
// outside; k_seg_jump then replaces flagged pointers by the label of their
// target, round after round (pointer doubling), until no flagged pointer is
// left.  The number of rounds is bounded; hitting the bound is reported as
// CWTHF_E_NOT_CONVERGED.  The result does not depend on update order: every
// update moves a pointer further along the (unique) chain.
#include "internal.cuh"

namespace cwthf {
namespace {

// Tile: kSegTX x kSegTY x kSegTZ owned cells.  A warp covers one grid row of
// 32 columns: lanes 1..30 own cells, lanes 0 and 31 read the x-halo columns.
// Warps 0 and 17 read the y-halo rows.
constexpr int kSegRows = kSegTY + 2;          // warps per CTA
constexpr int kSegThreads = 32 * kSegRows;    // 576
// Shared-memory parent pointers use a padded local index (lz * 16 + ly) * 32 + lx,
// so that local coordinates come back with shifts and masks.
constexpr int kPX = 32, kPXBits = 5;
constexpr int kPlaneL = kPX * kSegTY, kPlaneBits = 9;
constexpr int kLocal = kPlaneL * kSegTZ;  // 16384 entries
static_assert(kSegTX <= kPX && kPlaneL == (1 << kPlaneBits) && kSegTY == 16, "padded layout");
constexpr int32_t kFlag = 1 << 30;
constexpr int32_t kMask = kFlag - 1;
constexpr int kChaseLimit = 64;  // longest in-tile chain followed before handing over to the global pass
constexpr int kSegPrefetch = 4;  // planes of a column loaded ahead
// Seeds of one tile: at most one local maximum per 2 x 2 x 2 block of cells
// (any two cells of such a block are neighbours), so 15 * 8 * 16 per tile.
constexpr int kTileSeedCap = ((kSegTX + 1) / 2) * ((kSegTY + 1) / 2) * ((kSegTZ + 1) / 2);
constexpr int32_t kLocalMask = 0xffff;  // local index bits of a shared-memory pointer
constexpr int kCountShift = 16;         // a seed's in-tile cell count rides above them

__device__ __forceinline__ int wrap(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// Search codes of the three candidates (-1, 0, +1) along one axis: rank of
// the wrapped coordinate (0 = smallest) times 4 plus the candidate's position.
// The smallest code among the candidates holding the maximum is the winner
// under the strict order; kNoMatch (only reached when the window holds no
// comparable value, i.e. NaN input) decodes to the centre.
constexpr int kNoMatch = 13;
__device__ __forceinline__ void codes3(int m, int c, int p, int& km, int& kc, int& kp) {
    km = ((m > c) + (m > p)) * 4 + 0;
    kc = ((c > m) + (c > p)) * 4 + 1;
    kp = ((p > m) + (p > c)) * 4 + 2;
}

// Position (0, 1, 2 for -1, 0, +1) of the first candidate, in the strict
// order, whose value equals M.
__device__ __forceinline__ int pick3(float a, float b, float c, float M, int ka, int kb, int kc) {
    const int x = min(min(a == M ? ka : kNoMatch, b == M ? kb : kNoMatch), c == M ? kc : kNoMatch);
    return x & 3;
}

// Parents of a 30 x 16 x 32-cell tile and the in-tile part of every chain.
//
// The best of the 27 cells around c is found in two steps.  First the
// maximum value M, separably: along x by warp shuffles, along y through a
// shared buffer of x-window maxima, along z in registers over the last three
// planes.  Then the winner among the cells equal to M, which under the
// strict order is the one with the smallest wrapped (z, y, x) in
// lexicographic order: the first plane (in wrapped z order) whose window
// holds M, then in that plane the first row whose x-window holds M, then in
// that row the first column holding M.  Two rings of four planes in shared
// memory (raw values and x-window maxima) serve the search, so one barrier
// per plane suffices.  The parent is then formed without branches.  Parents
// go to shared memory; every cell then follows its chain there until it
// reaches a seed, a non-seed maximum, or a cell outside the tile.
__global__ void __launch_bounds__(kSegThreads, 2) k_seg_tile(const float* __restrict__ C, int ng, float cwt_min,
                                                         int32_t* __restrict__ label, uint32_t* __restrict__ seed_bits,
                                                         uint16_t* __restrict__ seed_cells, int* status) {
    extern __shared__ int32_t ptr[];  // [kLocal], dynamic
    __shared__ uint16_t tile_seeds[kTileSeedCap];
    __shared__ uint32_t n_tile_seeds;
    constexpr int kSlot = kSegRows * 32;          // floats per ring slot
    __shared__ float vals[4 * kSlot];             // raw values of planes p-3 .. p (ring)
    __shared__ float rmax[4 * kSlot];             // x-window maxima of the same planes
    const int ntx = (ng + kSegTX - 1) / kSegTX, nty = (ng + kSegTY - 1) / kSegTY;
    const int t = int(blockIdx.x);
    const int tx = t % ntx, ty = (t / ntx) % nty, tz = t / (ntx * nty);
    const int x0 = tx * kSegTX, y0 = ty * kSegTY, z0 = tz * kSegTZ;
    const int wx = min(kSegTX, ng - x0), wy = min(kSegTY, ng - y0), wz = min(kSegTZ, ng - z0);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned full = 0xffffffffu;
    // this lane's column and this warp's row (wrapped; columns past a small grid
    // need a full modulo)
    const int lx = lane - 1, ly = w - 1;  // owned local coordinates when in range
    const int xc = ((x0 + lx) % ng + ng) % ng, yc = ((y0 + ly) % ng + ng) % ng;
    const int xm = wrap(xc - 1, ng), xp = wrap(xc + 1, ng);
    const int ym = wrap(yc - 1, ng), yp = wrap(yc + 1, ng);
    const bool own = lx >= 0 && lx < wx && ly >= 0 && ly < wy;
    const bool row_warp = w >= 1 && w <= kSegTY;  // warps of owned rows (warp-uniform)
    int kxm, kxc, kxp, kym, kyc, kyp;
    codes3(xm, xc, xp, kxm, kxc, kxp);
    codes3(ym, yc, yp, kym, kyc, kyp);
    const int N = ng;
    const float* colp = C + size_t(yc) * N + xc;
    // search addresses stay inside the rows even for the two halo lanes
    const int lanec = min(max(lane, 1), 30);
    const float* rsrc = rmax + (w - 1) * 32 + lanec;
    const float* vsrc = vals + (w - 1) * 32 + lanec;
    const int i0 = ly * kPX + lx;

    bool bad = false;
    if (threadIdx.x == 0) n_tile_seeds = 0;  // ordered before its first use by the plane barriers
    float pl0 = 0.f, pl1 = 0.f, pl2 = 0.f;  // window maxima of planes p-2, p-1, p at this row and column
    // kSegPrefetch planes of this column in flight (a register ring), so that
    // the per-plane barrier does not expose the load latency
    static_assert(kSegPrefetch % 4 == 0, "ring slots follow the prefetch slot");
    const int np_ = wz + 2;
    const size_t plane = size_t(N) * N;
    float ring[kSegPrefetch];
#pragma unroll
    for (int d = 0; d < kSegPrefetch; d++)
        ring[d] = d < np_ ? __ldg(colp + size_t(wrap(z0 - 1 + d, ng)) * plane) : 0.f;
#pragma unroll 1
    for (int p0 = 0; p0 < np_; p0 += kSegPrefetch)
#pragma unroll
    for (int d = 0; d < kSegPrefetch; d++) {
        const int p = p0 + d;
        if (p >= np_) break;  // block-uniform
        const float v = ring[d];
        if (p + kSegPrefetch < np_) ring[d] = __ldg(colp + size_t(wrap(z0 - 1 + p + kSegPrefetch, ng)) * plane);
        bad |= (v != v);
        const float vl = __shfl_up_sync(full, v, 1), vr = __shfl_down_sync(full, v, 1);
        const int sp = d & 3;  // p & 3, since p0 is a multiple of 4 (folded once unrolled)
        vals[sp * kSlot + w * 32 + lane] = v;
        rmax[sp * kSlot + w * 32 + lane] = fmaxf(fmaxf(vl, v), vr);
        __syncthreads();
        if (!row_warp) continue;  // warp-uniform: halo-row warps only feed the buffers
        pl0 = pl1;
        pl1 = pl2;
        pl2 = fmaxf(fmaxf(rmax[sp * kSlot + (w - 1) * 32 + lane], rmax[sp * kSlot + w * 32 + lane]),
                    rmax[sp * kSlot + (w + 1) * 32 + lane]);
        if (p < 2) continue;  // block-uniform
        // the cell of plane p-1 (owned z index lz = p-2); z codes are uniform and
        // differ from the interior ones only on the two wrapped planes
        const int lz = p - 2;
        const int zc = z0 + lz;
        const bool zlo = zc == 0, zhi = zc == N - 1;
        const int kzm = zlo ? 8 : (zhi ? 4 : 0), kzc = zlo ? 1 : (zhi ? 9 : 5), kzp = zlo ? 6 : (zhi ? 2 : 10);
        const float M = fmaxf(fmaxf(pl0, pl1), pl2);
        const int cz = pick3(pl0, pl1, pl2, M, kzm, kzc, kzp);
        const int so = ((d + 2 + cz) & 3) * kSlot;  // ring slot of plane p-2+cz
        const int cy = pick3(rsrc[so], rsrc[so + 32], rsrc[so + 64], M, kym, kyc, kyp);
        const float* row = vsrc + so + cy * 32;
        const int cx = pick3(row[-1], row[0], row[1], M, kxm, kxc, kxp);
        const int i = i0 + lz * kPlaneL;
        const int dx = cx - 1, dy = cy - 1, dz = cz - 1;
        const bool is_max = (dx | dy | dz) == 0;
        const bool in_tile = unsigned(lx + dx) < unsigned(wx) && unsigned(ly + dy) < unsigned(wy) &&
                             unsigned(lz + dz) < unsigned(wz);
        const int gx = dx < 0 ? xm : (dx > 0 ? xp : xc);
        const int gy = dy < 0 ? ym : (dy > 0 ? yp : yc);
        const int gz = wrap(zc + dz, N);
        const int32_t outside = -2 - ((gz * N + gy) * N + gx);
        const bool seed = is_max && M > cwt_min;
        const int32_t val = is_max ? (seed ? i : -1) : (in_tile ? i + dx + dy * kPX + dz * kPlaneL : outside);
        if (own) {
            ptr[i] = val;
            if (seed) {
                const uint32_t g = uint32_t((zc * N + yc) * N + xc);
                atomicOr(&seed_bits[g >> 5], 1u << (g & 31));
                const uint32_t j = atomicAdd(&n_tile_seeds, 1u);
                if (j < uint32_t(kTileSeedCap)) tile_seeds[j] = uint16_t(i);
            }
        }
    }
    if (bad) set_status(status, CWTHF_E_BAD_INPUT);
    __syncthreads();

    // Follow each chain inside the tile.  A chain that ends at a seed of this
    // tile adds one to the seed's cell count, kept in the upper half of the
    // seed's own entry (its lower half stays its own index, so that every walk
    // still recognises it); the walked cell then points straight at the seed.
    // Every value read or written is a later point of the same chain, so
    // concurrent walks do not change any result.
    const int32_t gbase = (z0 * N + y0) * N + x0;
    if (own) {
        int32_t* out = label + (size_t(z0) * N + yc) * N + xc;
        for (int lz = 0; lz < wz; lz++, out += plane) {
            const int i = i0 + lz * kPlaneL;
            const int32_t v = ptr[i];
            int32_t cur = v >= 0 ? (v & kLocalMask) : v;
            int steps = 0;
            while (cur >= 0 && steps < kChaseLimit) {
                const int32_t nv = ptr[cur];
                const int32_t nxt = nv >= 0 ? (nv & kLocalMask) : nv;
                if (nxt == cur) break;  // a seed
                cur = nxt;
                steps++;
            }
            int32_t res;
            if (cur == -1) {
                res = -1;
            } else if (cur <= -2) {
                res = (-2 - cur) | kFlag;
            } else {
                const int px = cur & (kPX - 1), py = (cur >> kPXBits) & (kSegTY - 1), pz = cur >> kPlaneBits;
                const int32_t g = gbase + (pz * N + py) * N + px;
                const int32_t nv = ptr[cur];
                if (nv >= 0 && (nv & kLocalMask) == cur) {
                    res = g;
                    atomicAdd(&ptr[cur], 1 << kCountShift);
                } else {
                    res = g | kFlag;  // walk stopped at the limit: resume globally
                }
                if (steps > 1) ptr[i] = cur;  // i is not a seed here: its entry holds no count
            }
            *out = res;
        }
    }
    __syncthreads();
    // in-tile cell counts of this tile's seeds (cells reaching them from other
    // tiles are added by the global pass)
    const uint32_t nts = n_tile_seeds;
    if (threadIdx.x == 0 && nts > uint32_t(kTileSeedCap)) set_status(status, CWTHF_E_BAD_INPUT);
    for (uint32_t j = threadIdx.x; j < min(nts, uint32_t(kTileSeedCap)); j += blockDim.x) {
        const int i = tile_seeds[j];
        const int px = i & (kPX - 1), py = (i >> kPXBits) & (kSegTY - 1), pz = i >> kPlaneBits;
        seed_cells[size_t(gbase + (pz * N + py) * N + px)] = uint16_t(uint32_t(ptr[i]) >> kCountShift);
    }
}

// Finishes every flagged label by following its chain through the label
// grid (at most kChaseLimit steps per cell) and adds the cells of every seed
// that the tile pass could not count (those that arrived flagged).  Each warp
// takes 128 consecutive labels, queues its flagged ones in shared memory and
// chases them with all lanes at once, then counts the finished ones with one
// atomic per distinct seed among them.  Labels read while other threads update
// them are always a later point of the same chain, so the result does not
// depend on timing.  A cell still unfinished at the limit stays flagged
// (pointing further along) and sets changed[0]: the doubling rounds then
// finish it and the cells are recounted.
constexpr int kResolveThreads = 256;
__global__ void __launch_bounds__(kResolveThreads) k_seg_resolve(int32_t* __restrict__ label, int64_t cells,
                                                                 const uint32_t* __restrict__ bits,
                                                                 const uint32_t* __restrict__ prefix,
                                                                 const uint32_t* __restrict__ n_slots, HaloAcc* acc,
                                                                 int* __restrict__ changed) {
    __shared__ int32_t queue[kResolveThreads / 32][128];
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    int32_t* wq = queue[threadIdx.x >> 5];
    bool left = false;
    const int64_t n4 = (cells + 3) / 4;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t base = int64_t(blockIdx.x) * blockDim.x + (threadIdx.x & ~31); base < n4; base += stride) {
        const int64_t i = base + lane;  // warp-uniform trip count
        int v[4] = {-1, -1, -1, -1};
        const bool vec = 4 * i + 3 < cells;
        if (i < n4) {
            if (vec) {
                const int4 q = reinterpret_cast<const int4*>(label)[i];
                v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
            } else {
                for (int j = 0; j < 4 && 4 * i + j < cells; j++) v[j] = label[4 * i + j];
            }
        }
        // queue the flagged labels of the warp, in (j, lane) order
        bool fl[4];
        int pos[4];
        int total = 0;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            fl[j] = v[j] >= 0 && (v[j] & kFlag);
            const unsigned b = __ballot_sync(full, fl[j]);
            pos[j] = total + __popc(b & below);
            total += __popc(b);
            if (fl[j]) wq[pos[j]] = v[j];
        }
        if (total == 0) continue;  // warp-uniform
        __syncwarp();
        for (int e = lane; e < total; e += 32) {
            int32_t w = wq[e];
            int steps = 0;
            while (w >= 0 && (w & kFlag) && steps < kChaseLimit) {
                w = label[w & kMask];
                steps++;
            }
            wq[e] = w;
            left |= (w >= 0 && (w & kFlag));
        }
        __syncwarp();
        bool mine = false;
#pragma unroll
        for (int j = 0; j < 4; j++)
            if (fl[j]) {
                v[j] = wq[pos[j]];
                mine = true;
            }
        if (mine) {
            if (vec) reinterpret_cast<int4*>(label)[i] = make_int4(v[0], v[1], v[2], v[3]);
            else
                for (int j = 0; j < 4 && 4 * i + j < cells; j++) label[4 * i + j] = v[j];
        }
        // cells per seed among the finished queue entries: one atomic per distinct seed
        for (int e0 = 0; e0 < total; e0 += 32) {  // warp-uniform
            const int e = e0 + lane;
            int32_t lab = e < total ? wq[e] : -1;
            if (lab < 0 || (lab & kFlag)) lab = -1;
            const unsigned peers = __match_any_sync(full, lab);
            uint32_t slot;
            if (lab >= 0 && lane == __ffs(peers) - 1 && seed_slot(bits, prefix, n_slots, lab, slot))
                atomicAdd(&acc[slot].n_cells, (unsigned long long)__popc(peers));
        }
        __syncwarp();  // the queue is refilled next
    }
    if (__any_sync(full, left) && lane == 0) changed[0] = 1;
}

// Fallback when a chain outlived the bounded walks: after the doubling rounds,
// clear and recount the cells of every seed (does nothing otherwise).
__global__ void __launch_bounds__(256) k_seg_recount(const int32_t* __restrict__ label, int64_t cells,
                                                     const uint32_t* __restrict__ bits,
                                                     const uint32_t* __restrict__ prefix,
                                                     const uint32_t* __restrict__ n_slots, HaloAcc* acc,
                                                     const int* __restrict__ changed, int phase) {
    if (changed[0] == 0) return;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    const int64_t gid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (phase == 0) {
        for (int64_t s = gid; s < int64_t(*n_slots); s += stride) acc[s].n_cells = 0;
        return;
    }
    for (int64_t c = gid; c < cells; c += stride) {
        uint32_t slot;
        const int32_t l = label[c];
        if (l >= 0 && seed_slot(bits, prefix, n_slots, l, slot)) atomicAdd(&acc[slot].n_cells, 1ull);
    }
}

// One global round: replace every flagged pointer by its target's label;
// changed[round] records whether any pointer is still flagged afterwards.
__global__ void __launch_bounds__(kSegThreads) k_seg_jump(int32_t* __restrict__ label, int64_t cells,
                                                         int* __restrict__ changed, int round) {
    if (round > 0 && changed[round - 1] == 0) return;  // converged earlier
    bool any = false;
    int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; c < cells; c += stride) {
        int32_t v = label[c];
        if (v >= 0 && (v & kFlag)) {
            int32_t w = label[v & kMask];
            label[c] = w;
            any |= (w >= 0 && (w & kFlag));  // still a pointer: another round is needed
        }
    }
    if (__any_sync(0xffffffffu, any) && (threadIdx.x & 31) == 0) changed[round] = 1;
}

__global__ void k_seg_jump_check(const int* changed, int rounds, int* status) {
    if (changed[rounds - 1]) set_status(status, CWTHF_E_NOT_CONVERGED);
}

__global__ void k_popc(const uint32_t* __restrict__ bits, int64_t nwords, uint32_t* __restrict__ out) {
    int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < nwords; i += stride) out[i] = __popc(bits[i]);
}

// slot -> seed cell, in increasing cell order; clears the slot's accumulators
// (the cell count starts from the tile pass's in-tile count when given).
// *n_slots = number of seeds, clamped to slot_cap (more seeds than that can
// only come from an inconsistent label grid, reported as bad input).
__global__ void k_seed_list(const uint32_t* __restrict__ bits, const uint32_t* __restrict__ prefix, int64_t nwords,
                            int64_t slot_cap, int32_t* __restrict__ seed_list, const uint16_t* __restrict__ seed_cells,
                            HaloAcc* __restrict__ acc, uint32_t* __restrict__ n_slots, int* status) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        uint32_t total = prefix[nwords];
        if (int64_t(total) > slot_cap) set_status(status, CWTHF_E_BAD_INPUT);
        *n_slots = uint32_t(min(int64_t(total), slot_cap));
    }
    int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < nwords; i += stride) {
        uint32_t b = bits[i];
        uint32_t s = prefix[i];
        while (b && int64_t(s) < slot_cap) {
            int bit = __ffs(b) - 1;
            b &= b - 1;
            seed_list[s] = int32_t(i * 32 + bit);
            HaloAcc z;
            z.n_part = 0;
            z.mq = 0;
            z.mom[0] = z.mom[1] = z.mom[2] = 0;
            z.n_cells = seed_cells ? seed_cells[i * 32 + bit] : 0;
            acc[s] = z;
            s++;
        }
    }
}

// Seeds from a label grid: the cells labelled with their own index.
__global__ void k_seeds_from_labels(const int32_t* __restrict__ label, int64_t cells, uint32_t* __restrict__ bits,
                                    int* status) {
    int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; c < cells; c += stride) {
        int32_t l = label[c];
        if (l < -1 || l >= cells) set_status(status, CWTHF_E_BAD_INPUT);
        if (l == c) atomicOr(&bits[c >> 5], 1u << (c & 31));
    }
}

}  // namespace

int seeds_rank(cwthf_ctx* ctx, int ng, const uint16_t* seed_cells, cudaStream_t s) {
    int64_t cells = int64_t(ng) * ng * ng;
    int64_t nwords = (cells + 31) / 32;
    int blocks = ctx->sm_count * 8;
    CWTHF_LAUNCH(ctx, s, "k_popc", k_popc<<<blocks, 256, 0, s>>>(ctx->seed_bits, nwords, ctx->seed_prefix));
    int rc = scan_u32(ctx, ctx->seed_prefix, ctx->seed_prefix, nwords, s);
    if (rc) return rc;
    CWTHF_LAUNCH(ctx, s, "k_seed_list", k_seed_list<<<blocks, 256, 0, s>>>(ctx->seed_bits, ctx->seed_prefix, nwords, cells / 8 + 8, ctx->seed_list,
                                       seed_cells, ctx->acc, ctx->n_seeds, ctx->d_status));
    return cuda_status(cudaGetLastError());
}

int seeds_from_labels(cwthf_ctx* ctx, const int32_t* label, int ng, cudaStream_t s) {
    int64_t cells = int64_t(ng) * ng * ng;
    int64_t nwords = (cells + 31) / 32;
    cudaError_t e = cudaMemsetAsync(ctx->seed_bits, 0, size_t(nwords) * 4, s);
    if (e != cudaSuccess) return cuda_status(e);
    CWTHF_LAUNCH(ctx, s, "k_seeds_from_labels", k_seeds_from_labels<<<ctx->sm_count * 8, 256, 0, s>>>(label, cells, ctx->seed_bits, ctx->d_status));
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e);
    return seeds_rank(ctx, ng, nullptr, s);
}

int segment_impl(cwthf_ctx* ctx, const float* cwt, int ng, float cwt_min, int32_t* label, bool,
                 cudaStream_t s) {
    int64_t cells = int64_t(ng) * ng * ng;
    int64_t nwords = (cells + 31) / 32;
    cudaError_t e = cudaMemsetAsync(ctx->seed_bits, 0, size_t(nwords) * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->jump_changed, 0, sizeof(int) * (kMaxJumpRounds + 1), s);
    if (e != cudaSuccess) return cuda_status(e);
    int64_t ntiles = int64_t(div_up(ng, kSegTX)) * div_up(ng, kSegTY) * div_up(ng, kSegTZ);
    cudaFuncSetAttribute(k_seg_tile, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sizeof(int32_t) * kLocal));
    CWTHF_LAUNCH(ctx, s, "k_seg_tile",
                 k_seg_tile<<<unsigned(ntiles), kSegThreads, sizeof(int32_t) * kLocal, s>>>(cwt, ng, cwt_min, label,
                                                                                          ctx->seed_bits,
                                                                                          ctx->seed_cells,
                                                                                          ctx->d_status));
    // seed ranks first (the resolve pass counts cells per seed slot)
    int rc = seeds_rank(ctx, ng, ctx->seed_cells, s);
    if (rc) return rc;
    int blocks = ctx->sm_count * 8;
    CWTHF_LAUNCH(ctx, s, "k_seg_resolve",
                 k_seg_resolve<<<blocks, kResolveThreads, 0, s>>>(label, cells, ctx->seed_bits, ctx->seed_prefix, ctx->n_seeds,
                                                      ctx->acc, ctx->jump_changed));
    // pointer doubling for whatever the bounded walks left (normally nothing: every round exits at once)
    for (int r = 1; r < kMaxJumpRounds; r++) {
        CWTHF_LAUNCH(ctx, s, "k_seg_jump", k_seg_jump<<<blocks, 256, 0, s>>>(label, cells, ctx->jump_changed, r));
    }
    CWTHF_LAUNCH(ctx, s, "k_seg_jump_check", k_seg_jump_check<<<1, 1, 0, s>>>(ctx->jump_changed, kMaxJumpRounds, ctx->d_status));
    for (int phase = 0; phase < 2; phase++)
        CWTHF_LAUNCH(ctx, s, "k_seg_recount",
                     k_seg_recount<<<blocks, 256, 0, s>>>(label, cells, ctx->seed_bits, ctx->seed_prefix,
                                                          ctx->n_seeds, ctx->acc, ctx->jump_changed, phase));
    return cuda_status(cudaGetLastError());
}

}  // namespace cwthf
