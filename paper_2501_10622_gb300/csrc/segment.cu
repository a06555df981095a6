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
constexpr int kOwned = kSegTX * kSegTY * kSegTZ;
constexpr int32_t kFlag = 1 << 30;
constexpr int32_t kMask = kFlag - 1;
constexpr int kChaseLimit = 64;  // longest in-tile chain followed before handing over to the global pass
constexpr int kSegPrefetch = 8;  // planes of a column loaded ahead

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
// per plane suffices.  Parents go to shared memory; every cell then follows
// its chain there until it reaches a seed, a non-seed maximum, or a cell
// outside the tile.
__global__ void __launch_bounds__(kSegThreads, 2) k_seg_tile(const float* __restrict__ C, int ng, float cwt_min,
                                                         int32_t* __restrict__ label, uint32_t* __restrict__ seed_bits,
                                                         int* status) {
    extern __shared__ int32_t ptr[];  // [kOwned], dynamic
    __shared__ float vals[4][kSegRows][32];  // raw values of planes p-3 .. p (ring)
    __shared__ float rmax[4][kSegRows][32];  // x-window maxima of the same planes
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
    int kxm, kxc, kxp, kym, kyc, kyp;
    codes3(xm, xc, xp, kxm, kxc, kxp);
    codes3(ym, yc, yp, kym, kyc, kyp);
    const size_t N = size_t(ng);
    const float* colp = C + size_t(yc) * N + xc;

    bool bad = false;
    float pl0 = 0.f, pl1 = 0.f, pl2 = 0.f;  // window maxima of planes p-2, p-1, p at this row and column
    // kSegPrefetch planes of this column in flight (a register ring), so that
    // the per-plane barrier does not expose the load latency
    const int np_ = wz + 2;
    const size_t plane = N * N;
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
        const int sp = p & 3;
        vals[sp][w][lane] = v;
        rmax[sp][w][lane] = fmaxf(fmaxf(vl, v), vr);
        __syncthreads();
        if (w >= 1 && w <= kSegTY) {
            pl0 = pl1;
            pl1 = pl2;
            pl2 = fmaxf(fmaxf(rmax[sp][w - 1][lane], rmax[sp][w][lane]), rmax[sp][w + 1][lane]);
        }
        if (p >= 2 && own) {
            // the cell of plane p-1 (owned z index lz = p-2)
            const int lz = p - 2;
            const int zc = z0 + lz, zm = wrap(zc - 1, ng), zp = wrap(zc + 1, ng);
            int kzm, kzc, kzp;
            codes3(zm, zc, zp, kzm, kzc, kzp);
            const float M = fmaxf(fmaxf(pl0, pl1), pl2);
            const int cz = pick3(pl0, pl1, pl2, M, kzm, kzc, kzp);
            const int sz = (p - 2 + cz) & 3;
            const int cy = pick3(rmax[sz][w - 1][lane], rmax[sz][w][lane], rmax[sz][w + 1][lane], M, kym, kyc, kyp);
            const float* row = &vals[sz][w - 1 + cy][lane];
            const int cx = pick3(row[-1], row[0], row[1], M, kxm, kxc, kxp);
            const int i = (lz * kSegTY + ly) * kSegTX + lx;
            if (cx == 1 && cy == 1 && cz == 1) {
                // a local maximum: a seed iff its value > cwt_min
                if (M > cwt_min) {
                    ptr[i] = i;
                    const uint32_t g = uint32_t((size_t(zc) * N + yc) * N + xc);
                    atomicOr(&seed_bits[g >> 5], 1u << (g & 31));
                } else {
                    ptr[i] = -1;
                }
            } else {
                const int qx = lx + cx - 1, qy = ly + cy - 1, qz = lz + cz - 1;
                if (unsigned(qx) < unsigned(wx) && unsigned(qy) < unsigned(wy) && unsigned(qz) < unsigned(wz)) {
                    ptr[i] = i + (cx - 1) + (cy - 1) * kSegTX + (cz - 1) * (kSegTX * kSegTY);
                } else {
                    const int px = cx == 0 ? xm : (cx == 2 ? xp : xc);
                    const int py = cy == 0 ? ym : (cy == 2 ? yp : yc);
                    const int pz = cz == 0 ? zm : (cz == 2 ? zp : zc);
                    ptr[i] = -2 - int32_t((size_t(pz) * N + py) * N + px);
                }
            }
        }
    }
    if (bad) set_status(status, CWTHF_E_BAD_INPUT);
    __syncthreads();

    // follow each chain inside the tile (read-only walk over the parents)
    if (own) {
        int32_t* out = label + (size_t(z0) * N + yc) * N + xc;
        for (int lz = 0; lz < wz; lz++, out += N * N) {
            const int i = (lz * kSegTY + ly) * kSegTX + lx;
            int32_t cur = ptr[i];
            int steps = 0;
            while (cur >= 0 && steps < kChaseLimit) {
                const int32_t nxt = ptr[cur];
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
                const int px = cur % kSegTX, py = (cur / kSegTX) % kSegTY, pz = cur / (kSegTX * kSegTY);
                const int32_t g = int32_t((size_t(z0 + pz) * N + (y0 + py)) * N + (x0 + px));
                res = (ptr[cur] == cur) ? g : (g | kFlag);  // walk stopped at the limit: resume globally
            }
            *out = res;
        }
    }
}

// Finishes every flagged label by following its chain through the label
// grid (at most kChaseLimit steps per cell) and counts the cells of every
// seed.  Labels read while other threads update them are always a later point
// of the same chain, so the result does not depend on timing.  A cell still
// unfinished at the limit stays flagged (pointing further along) and sets
// changed[0]: the doubling rounds then finish it and the cells are recounted.
__global__ void __launch_bounds__(256) k_seg_resolve(int32_t* __restrict__ label, int64_t cells,
                                                     const uint32_t* __restrict__ bits,
                                                     const uint32_t* __restrict__ prefix,
                                                     const uint32_t* __restrict__ n_slots, HaloAcc* acc,
                                                     int* __restrict__ changed) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
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
        bool wrote = false;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            int32_t w = v[j];
            if (w < 0 || !(w & kFlag)) continue;
            int steps = 0;
            while (w >= 0 && (w & kFlag) && steps < kChaseLimit) {
                w = label[w & kMask];
                steps++;
            }
            v[j] = w;
            wrote = true;
            left |= (w >= 0 && (w & kFlag));
        }
        if (wrote) {
            if (vec) reinterpret_cast<int4*>(label)[i] = make_int4(v[0], v[1], v[2], v[3]);
            else
                for (int j = 0; j < 4 && 4 * i + j < cells; j++) label[4 * i + j] = v[j];
        }
        // cells per seed: runs of equal labels within the thread, one atomic per run,
        // or one per warp when all 128 labels of the warp are the same seed
        // (the shuffle runs on every lane: it must not sit behind a short-circuit)
        const int lead = __shfl_sync(full, v[3], 0);
        const bool same = (v[0] == v[3]) & (v[1] == v[3]) & (v[2] == v[3]) & (v[3] == lead);
        const bool uniform = __all_sync(full, same);
        if (uniform) {
            uint32_t slot;
            if (lane == 0 && v[0] >= 0 && !(v[0] & kFlag) && seed_slot(bits, prefix, n_slots, v[0], slot))
                atomicAdd(&acc[slot].n_cells, 128ull);  // padding entries are -1, so all 128 are cells
        } else {
            int j = 0;
            while (j < 4) {
                int k = j + 1;
                while (k < 4 && v[k] == v[j]) k++;
                uint32_t slot;
                if (v[j] >= 0 && !(v[j] & kFlag) && seed_slot(bits, prefix, n_slots, v[j], slot))
                    atomicAdd(&acc[slot].n_cells, (unsigned long long)(k - j));
                j = k;
            }
        }
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

// slot -> seed cell, in increasing cell order; clears the slot's accumulators.
// *n_slots = number of seeds, clamped to slot_cap (more seeds than that can
// only come from an inconsistent label grid, reported as bad input).
__global__ void k_seed_list(const uint32_t* __restrict__ bits, const uint32_t* __restrict__ prefix, int64_t nwords,
                            int64_t slot_cap, int32_t* __restrict__ seed_list, HaloAcc* __restrict__ acc,
                            uint32_t* __restrict__ n_slots, int* status) {
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
            z.n_cells = 0;
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

int seeds_rank(cwthf_ctx* ctx, int ng, cudaStream_t s) {
    int64_t cells = int64_t(ng) * ng * ng;
    int64_t nwords = (cells + 31) / 32;
    int blocks = ctx->sm_count * 8;
    CWTHF_LAUNCH(ctx, s, "k_popc", k_popc<<<blocks, 256, 0, s>>>(ctx->seed_bits, nwords, ctx->seed_prefix));
    int rc = scan_u32(ctx, ctx->seed_prefix, ctx->seed_prefix, nwords, s);
    if (rc) return rc;
    CWTHF_LAUNCH(ctx, s, "k_seed_list", k_seed_list<<<blocks, 256, 0, s>>>(ctx->seed_bits, ctx->seed_prefix, nwords, cells / 8 + 8, ctx->seed_list,
                                       ctx->acc, ctx->n_seeds, ctx->d_status));
    return cuda_status(cudaGetLastError());
}

int seeds_from_labels(cwthf_ctx* ctx, const int32_t* label, int ng, cudaStream_t s) {
    int64_t cells = int64_t(ng) * ng * ng;
    int64_t nwords = (cells + 31) / 32;
    cudaError_t e = cudaMemsetAsync(ctx->seed_bits, 0, size_t(nwords) * 4, s);
    if (e != cudaSuccess) return cuda_status(e);
    CWTHF_LAUNCH(ctx, s, "k_seeds_from_labels", k_seeds_from_labels<<<ctx->sm_count * 8, 256, 0, s>>>(label, cells, ctx->seed_bits, ctx->d_status));
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e);
    return seeds_rank(ctx, ng, s);
}

int segment_impl(cwthf_ctx* ctx, const float* cwt, int ng, float cwt_min, int32_t* label, bool,
                 cudaStream_t s) {
    int64_t cells = int64_t(ng) * ng * ng;
    int64_t nwords = (cells + 31) / 32;
    cudaError_t e = cudaMemsetAsync(ctx->seed_bits, 0, size_t(nwords) * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->jump_changed, 0, sizeof(int) * (kMaxJumpRounds + 1), s);
    if (e != cudaSuccess) return cuda_status(e);
    int64_t ntiles = int64_t(div_up(ng, kSegTX)) * div_up(ng, kSegTY) * div_up(ng, kSegTZ);
    cudaFuncSetAttribute(k_seg_tile, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sizeof(int32_t) * kOwned));
    CWTHF_LAUNCH(ctx, s, "k_seg_tile",
                 k_seg_tile<<<unsigned(ntiles), kSegThreads, sizeof(int32_t) * kOwned, s>>>(cwt, ng, cwt_min, label,
                                                                                          ctx->seed_bits,
                                                                                          ctx->d_status));
    // seed ranks first (the resolve pass counts cells per seed slot)
    int rc = seeds_rank(ctx, ng, s);
    if (rc) return rc;
    int blocks = ctx->sm_count * 8;
    CWTHF_LAUNCH(ctx, s, "k_seg_resolve",
                 k_seg_resolve<<<blocks, 256, 0, s>>>(label, cells, ctx->seed_bits, ctx->seed_prefix, ctx->n_seeds,
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
