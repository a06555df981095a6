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

constexpr int kSegThreads = 256;
constexpr int kHX = kSegTX + 2, kHY = kSegTY + 2, kHZ = kSegTZ + 2;
constexpr int kOwned = kSegTX * kSegTY * kSegTZ;
constexpr int32_t kFlag = 1 << 30;
constexpr int32_t kMask = kFlag - 1;
constexpr int kLocalRounds = 12;  // > log2(kOwned) + 1

__device__ __forceinline__ bool beats(float va, int64_t ia, float vb, int64_t ib) {
    return va > vb || (va == vb && ia < ib);
}

__global__ void __launch_bounds__(kSegThreads) k_seg_tile(const float* __restrict__ C, int ng, float cwt_min,
                                                         int32_t* __restrict__ label, uint32_t* __restrict__ seed_bits,
                                                         int* status) {
    __shared__ float h[kHZ][kHY][kHX];
    __shared__ int32_t ptr[kOwned];
    const int ntx = (ng + kSegTX - 1) / kSegTX, nty = (ng + kSegTY - 1) / kSegTY;
    const int64_t t = blockIdx.x;
    const int tx = int(t % ntx), ty = int((t / ntx) % nty), tz = int(t / (int64_t(ntx) * nty));
    const int x0 = tx * kSegTX, y0 = ty * kSegTY, z0 = tz * kSegTZ;
    const int wx = min(kSegTX, ng - x0), wy = min(kSegTY, ng - y0), wz = min(kSegTZ, ng - z0);
    const int64_t N = ng;

    bool bad = false;
    for (int i = threadIdx.x; i < kHX * kHY * kHZ; i += kSegThreads) {
        int hx = i % kHX, hy = (i / kHX) % kHY, hz = i / (kHX * kHY);
        float v = -INFINITY;
        if (hx <= wx + 1 && hy <= wy + 1 && hz <= wz + 1) {
            int gx = x0 - 1 + hx, gy = y0 - 1 + hy, gz = z0 - 1 + hz;
            gx = gx < 0 ? gx + ng : (gx >= ng ? gx - ng : gx);
            gy = gy < 0 ? gy + ng : (gy >= ng ? gy - ng : gy);
            gz = gz < 0 ? gz + ng : (gz >= ng ? gz - ng : gz);
            v = C[(gz * N + gy) * N + gx];
            bad |= (v != v);
        }
        h[hz][hy][hx] = v;
    }
    if (bad) set_status(status, CWTHF_E_BAD_INPUT);
    __syncthreads();

    // parents of the owned cells
    for (int i = threadIdx.x; i < kOwned; i += kSegThreads) {
        int lx = i % kSegTX, ly = (i / kSegTX) % kSegTY, lz = i / (kSegTX * kSegTY);
        if (lx >= wx || ly >= wy || lz >= wz) { ptr[i] = -1; continue; }
        int bx = 0, by = 0, bz = 0;
        int gx0 = x0 + lx, gy0 = y0 + ly, gz0 = z0 + lz;
        float bv = h[lz + 1][ly + 1][lx + 1];
        int64_t bi = (gz0 * N + gy0) * N + gx0;
#pragma unroll
        for (int dz = -1; dz <= 1; dz++)
#pragma unroll
            for (int dy = -1; dy <= 1; dy++)
#pragma unroll
                for (int dx = -1; dx <= 1; dx++) {
                    if (dx == 0 && dy == 0 && dz == 0) continue;
                    float v = h[lz + 1 + dz][ly + 1 + dy][lx + 1 + dx];
                    if (v < bv) continue;  // cannot beat (fast path; ties fall through)
                    int gx = gx0 + dx, gy = gy0 + dy, gz = gz0 + dz;
                    gx = gx < 0 ? gx + ng : (gx >= ng ? gx - ng : gx);
                    gy = gy < 0 ? gy + ng : (gy >= ng ? gy - ng : gy);
                    gz = gz < 0 ? gz + ng : (gz >= ng ? gz - ng : gz);
                    int64_t gi = (gz * N + gy) * N + gx;
                    if (beats(v, gi, bv, bi)) {
                        bv = v;
                        bi = gi;
                        bx = dx;
                        by = dy;
                        bz = dz;
                    }
                }
        if (bx == 0 && by == 0 && bz == 0) {
            // a local maximum: a seed if above cwt_min, otherwise a root labelled -1
            if (bv > cwt_min) {
                ptr[i] = i;
                atomicOr(&seed_bits[bi >> 5], 1u << (bi & 31));
            } else {
                ptr[i] = -1;
            }
        } else {
            int gx = int(bi % N), gy = int((bi / N) % N), gz = int(bi / (N * N));
            int px = gx - x0, py = gy - y0, pz = gz - z0;
            if (px >= 0 && px < wx && py >= 0 && py < wy && pz >= 0 && pz < wz)
                ptr[i] = (pz * kSegTY + py) * kSegTX + px;
            else
                ptr[i] = -2 - int32_t(bi);
        }
    }
    __syncthreads();

    // pointer jumping inside the tile
    for (int round = 0; round < kLocalRounds; round++) {
        bool changed = false;
        for (int i = threadIdx.x; i < kOwned; i += kSegThreads) {
            int32_t p = ptr[i];
            if (p >= 0 && p != i) {
                int32_t q = ptr[p];
                if (q != p) {
                    ptr[i] = q;
                    changed = true;
                }
            }
        }
        if (!__syncthreads_or(changed)) break;
    }

    for (int i = threadIdx.x; i < kOwned; i += kSegThreads) {
        int lx = i % kSegTX, ly = (i / kSegTX) % kSegTY, lz = i / (kSegTX * kSegTY);
        if (lx >= wx || ly >= wy || lz >= wz) continue;
        int32_t p = ptr[i], out;
        if (p == -1) {
            out = -1;
        } else if (p <= -2) {
            out = (-2 - p) | kFlag;
        } else {
            int px = p % kSegTX, py = (p / kSegTX) % kSegTY, pz = p / (kSegTX * kSegTY);
            int32_t g = int32_t(((z0 + pz) * N + (y0 + py)) * N + (x0 + px));
            out = (ptr[p] == p) ? g : (g | kFlag);  // not yet resolved only if the local bound was hit
        }
        label[((z0 + lz) * N + (y0 + ly)) * N + (x0 + lx)] = out;
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
    CWTHF_LAUNCH(ctx, s, "k_seg_tile", k_seg_tile<<<unsigned(ntiles), kSegThreads, 0, s>>>(cwt, ng, cwt_min, label, ctx->seed_bits, ctx->d_status));
    int blocks = ctx->sm_count * 8;
    for (int r = 0; r < kMaxJumpRounds; r++) {
        CWTHF_LAUNCH(ctx, s, "k_seg_jump", k_seg_jump<<<blocks, kSegThreads, 0, s>>>(label, cells, ctx->jump_changed, r));
    }
    CWTHF_LAUNCH(ctx, s, "k_seg_jump_check", k_seg_jump_check<<<1, 1, 0, s>>>(ctx->jump_changed, kMaxJumpRounds, ctx->d_status));
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e);
    return seeds_rank(ctx, ng, s);
}

}  // namespace cwthf
