// segment.cu -- local maxima and steepest-ascent segmentation of the CWT field
// (Sec. 2 steps 4-5, Sec. 2.3).
//
// Order on cells: a beats b iff C[a] > C[b], or C[a] == C[b] and a < b
// (a, b linear indices).  parent(c) = the best of c and its 26 periodic
// neighbours; c is a local maximum iff parent(c) == c.  A maximum with
// C > cwt_min is a seed; the label of a cell is the seed its parent chain
// reaches, or -1 when the chain ends at a maximum that is not a seed.
//
// k_seg_parent finds every cell's parent and writes it as a one-byte code
// (the offset along each axis, a maximum flag, a seed flag): each thread keeps
// a column of rows in registers and walks along z, so the 27-cell search needs
// no shared memory and no barrier.  k_seg_chase loads a tile's codes into
// shared memory as parent pointers and resolves every chain that stays inside
// the tile.  A chain that leaves the tile is written as a flagged pointer
// (-2 - g) to the first cell g outside; the global pass then replaces flagged
// pointers by the label of their target (bounded walks, then, only if a chain
// outlived them, pointer-doubling rounds in one cooperative launch; hitting the
// round bound is reported as CWTHF_E_NOT_CONVERGED).  The result does not
// depend on update order: every update moves a pointer further along the
// (unique) chain.
#include <cuda/atomic>
#include <type_traits>

#include "internal.cuh"

namespace cwthf {
namespace {

// Chain tiles: 64 x 16 x 16 cells, one warp per row of 64 columns, each lane
// owning two adjacent columns (one 2-byte code load, one 8-byte pointer and
// label store per cell pair).  Shared parent pointers use the local index
// (lz * 16 + ly) * 64 + lx, so local coordinates come back with shifts and
// masks.  A tile row's flagged cells go out as 32 masks: word 2 lz + p holds
// plane lz's columns of parity p (bit = lane).
constexpr int kChTX = 64, kChTY = 16, kChTZ = 16;
constexpr int kChThreads = 32 * kChTY;  // 512
constexpr int kPX = 64, kPXBits = 6;
constexpr int kPlaneL = kPX * kChTY, kPlaneBits = 10;
constexpr int kLocal = kPlaneL * kChTZ;  // 16384 entries
constexpr int kRowWords = 2 * kChTZ;     // flagged-cell masks per tile row (32)
static_assert(kChTX == kPX && kPlaneL == (1 << kPlaneBits) && kRowWords == 32, "local index layout");
// A flagged pointer (a chain still to be followed) to cell g is stored as
// -2 - g, apart from -1 (no seed) and the final labels (seed cells, >= 0).
__device__ __forceinline__ bool is_flagged(int32_t v) { return v <= -2; }
__device__ __forceinline__ int32_t flag_target(int32_t v) { return -2 - v; }
constexpr int kJumpRoundsInTile = 16;  // in-place jumping rounds (each at least doubles the distance): 2^14 >= cells of a tile
// Seeds of one tile: at most one local maximum per 2 x 2 x 2 block of cells
// (any two cells of such a block are neighbours).
constexpr int kTileSeedCap = (kChTX / 2) * (kChTY / 2) * (kChTZ / 2);
constexpr int32_t kLocalMask = 0xffff;  // local index bits of a shared-memory pointer
constexpr int kCountShift = 16;         // a seed's in-tile cell count rides above them

// Parent codes: bits 0-1 / 2-3 / 4-5 the offset + 1 along x / y / z; a local
// maximum has offsets (0, 0, 0); bit 6 marks a maximum that seeds a halo.
constexpr uint8_t kCodeMax = 0x15, kCodeSeed = 0x40;

// Parent-code blocks: a warp owns 30 columns (lanes 1-30; lanes 0 and 31 hold
// the x-halo columns) x kParR rows (plus the two y-halo rows) x kParZ planes
// (plus one halo plane at each end), streamed through a ring of kParStages
// planes in shared memory.
constexpr int kParR = 4, kParZ = 128, kParWarps = 4, kParStages = 6, kParBlocks = 6;
constexpr int kParThreads = 32 * kParWarps;

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
// Winner of a window of three candidates along one axis (offsets -1, 0, +1),
// with their window maxima a, b, c and payloads qa, qb, qc (the choices made
// along the axes searched before this one); the winner's choice (0, 1, 2) is
// added to its payload at bit `shift`.  Away from the periodic boundary (I) the
// strict order ranks the candidates in position order, so the winner is the
// first one holding the maximum: a later candidate wins only if strictly
// greater.  At the boundary the search codes of the wrapped coordinates decide.
template <bool I>
__device__ __forceinline__ void win3(float a, float b, float c, uint32_t qa, uint32_t qb, uint32_t qc, int ka, int kb,
                                     int kc, int shift, float& m, uint32_t& q) {
    if (I) {
        const float m1 = fmaxf(a, b);
        const uint32_t q1 = b > a ? (qb | (1u << shift)) : qa;
        m = fmaxf(m1, c);
        q = c > m1 ? (qc | (2u << shift)) : q1;
    } else {
        m = fmaxf(fmaxf(a, b), c);
        const int k = pick3(a, b, c, m, ka, kb, kc);
        q = (k == 0 ? qa : (k == 1 ? qb : qc)) | (uint32_t(k) << shift);
    }
}

// Asynchronous 4-byte copy global -> shared (sm_80+ cp.async), completed in
// groups: each thread waits only for its own copies.
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(uint32_t(__cvta_generic_to_shared(dst))),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Parent code of every cell.  The best of the 27 cells around c is the first
// cell, in wrapped (z, y, x) lexicographic order, holding the window's maximum
// M, so it is found separably: per row and plane the x window (warp shuffles)
// gives the row's maximum and x choice; per plane the y window over the
// thread's rows gives the plane's maximum and (y, x) choice; the z window over
// a ring of the last three planes gives M and the full choice, which is the
// parent code itself (offset + 1 along x, y, z in bits 0-1, 2-3, 4-5).  The
// choices ride along with the maxima as payloads, so no choice is searched for
// twice.  Each lane streams its column's rows through a ring of kParStages
// planes in shared memory (asynchronous copies issued kParStages - 1 planes
// ahead), which keeps enough loads in flight without holding them in
// registers.  The plane loop is unrolled six times, so that the ring slots
// rotate by renaming rather than copying.
// One warp's block.  XI / YI: the block's owned columns / rows are away from
// the periodic boundary, where the x / y choices reduce to position order;
// the z choice takes the same shortcut on every plane but the two wrapped ones.
template <bool XI, bool YI>
__device__ __forceinline__ void parent_block(const float* __restrict__ C, int N, float cwt_min,
                                             uint8_t* __restrict__ code_out, uint32_t* __restrict__ seed_bits,
                                             int* status, int x0, int y0, int z0, int wzc, float* ring) {
    constexpr int R = kParR, NR = kParR + 2, S = kParStages;
    static_assert(6 % S == 0, "the unrolled loop fixes each plane's ring slot");
    const int lane = threadIdx.x & 31;
    const unsigned full = 0xffffffffu;
    const int xc = ((x0 + lane - 1) % N + N) % N;
    const bool own_x = lane >= 1 && lane <= 30 && x0 + lane - 1 < N;
    int kxm = 0, kxc = 5, kxp = 10;
    if (!XI) codes3(wrap(xc - 1, N), xc, wrap(xc + 1, N), kxm, kxc, kxp);
    // offsets of the rows y0-1 .. y0+R (wrapped) and the y search codes of the
    // owned rows, packed km | kc << 4 | kp << 8 per row
    int32_t yoff[NR];
#pragma unroll
    for (int j = 0; j < NR; j++) yoff[j] = (((y0 - 1 + j) % N + N) % N) * N;
    int ykc[R];
#pragma unroll
    for (int r = 0; r < R; r++) {
        ykc[r] = 0 | (5 << 4) | (10 << 8);
        if (!YI) {
            int a, b, c;
            codes3(yoff[r] / N, yoff[r + 1] / N, yoff[r + 2] / N, a, b, c);
            ykc[r] = a | (b << 4) | (c << 8);
        }
    }
    const int32_t plane = N * N;
    const float* colp = C + xc;
    const int np_ = wzc + 2;
    float* my = ring + lane;  // this lane's column of ring slot s, row j: my[(s * NR + j) * 32]
    // copies of plane p (z = z0 - 1 + p, wrapped) into ring slot p % S, one group per plane
    auto issue = [&](int p) {
        if (p < np_) {
            const int z = ((z0 - 1 + p) % N + N) % N;
            const float* base = colp + size_t(z) * size_t(plane);
            float* dst = my + (p % S) * NR * 32;
#pragma unroll
            for (int j = 0; j < NR; j++) cp_async4(dst + j * 32, base + yoff[j]);
        }
        cp_async_commit();  // empty groups past the end keep the count uniform
    };
    bool bad = false;
    // plane p (ring slot p % S, unroll position u = p % 6): x and y windows
    // into the window ring slot (mn, qn), then the z windows of plane p - 1
    // from the slots of planes p - 2 (mo, qo), p - 1 (mm, qm) and p (mn, qn)
    auto step = [&](int p, auto u, const float (&mo)[R], const uint32_t (&qo)[R], const float (&mm)[R],
                    const uint32_t (&qm)[R], float (&mn)[R], uint32_t (&qn)[R]) {
        issue(p + S - 1);
        cp_async_wait<S - 1>();  // this lane's copies of plane p have landed
        const float* src = my + (decltype(u)::value % S) * NR * 32;
        float rm[NR];
        uint32_t rq[NR];
#pragma unroll
        for (int j = 0; j < NR; j++) {
            const float v = src[j * 32];
            bad |= (v != v);
            const float vl = __shfl_up_sync(full, v, 1), vr = __shfl_down_sync(full, v, 1);
            win3<XI>(vl, v, vr, 0u, 0u, 0u, kxm, kxc, kxp, 0, rm[j], rq[j]);
        }
#pragma unroll
        for (int r = 0; r < R; r++)
            win3<YI>(rm[r], rm[r + 1], rm[r + 2], rq[r], rq[r + 1], rq[r + 2], ykc[r] & 15, (ykc[r] >> 4) & 15,
                     ykc[r] >> 8, 2, mn[r], qn[r]);
        if (p >= 2) {
            // the cells of plane p-1 (z = z0 + p - 2)
            const int zc = z0 + p - 2;
            const bool zlo = zc == 0, zhi = zc == N - 1;
            const int kzm = zlo ? 8 : (zhi ? 4 : 0), kzc = zlo ? 1 : (zhi ? 9 : 5), kzp = zlo ? 6 : (zhi ? 2 : 10);
            uint8_t* out = code_out + size_t(zc) * size_t(plane) + xc;
            const int32_t gz = zc * plane + xc;
            auto emit = [&](auto zi) {
#pragma unroll
                for (int r = 0; r < R; r++) {
                    float M;
                    uint32_t code;
                    win3<decltype(zi)::value>(mo[r], mm[r], mn[r], qo[r], qm[r], qn[r], kzm, kzc, kzp, 4, M, code);
                    const bool seed = code == kCodeMax && M > cwt_min;
                    if (own_x && y0 + r < N) {
                        out[yoff[r + 1]] = uint8_t(code | (seed ? kCodeSeed : 0u));
                        if (seed) {
                            const uint32_t g = uint32_t(gz + yoff[r + 1]);
                            atomicOr(&seed_bits[g >> 5], 1u << (g & 31));
                        }
                    }
                }
            };
            if (!zlo && !zhi) emit(std::integral_constant<bool, true>{});  // uniform: once per plane
            else emit(std::integral_constant<bool, false>{});
        }
    };
    float m0[R], m1[R], m2[R];
    uint32_t q0[R], q1[R], q2[R];
#pragma unroll
    for (int p = 0; p < S - 1; p++) issue(p);
    // plane p goes to window ring slot p % 3
#pragma unroll 1
    for (int p = 0; p < np_; p += 6) {
        using I0 = std::integral_constant<int, 0>;
        using I1 = std::integral_constant<int, 1>;
        using I2 = std::integral_constant<int, 2>;
        using I3 = std::integral_constant<int, 3>;
        using I4 = std::integral_constant<int, 4>;
        using I5 = std::integral_constant<int, 5>;
        step(p, I0{}, m1, q1, m2, q2, m0, q0);
        if (p + 1 >= np_) break;
        step(p + 1, I1{}, m2, q2, m0, q0, m1, q1);
        if (p + 2 >= np_) break;
        step(p + 2, I2{}, m0, q0, m1, q1, m2, q2);
        if (p + 3 >= np_) break;
        step(p + 3, I3{}, m1, q1, m2, q2, m0, q0);
        if (p + 4 >= np_) break;
        step(p + 4, I4{}, m2, q2, m0, q0, m1, q1);
        if (p + 5 >= np_) break;
        step(p + 5, I5{}, m0, q0, m1, q1, m2, q2);
    }
    cp_async_wait<0>();  // nothing left in flight (the trailing groups are empty)
    if (bad) set_status(status, CWTHF_E_BAD_INPUT);
}

__global__ void __launch_bounds__(kParThreads, kParBlocks) k_seg_parent(const float* __restrict__ C, int ng,
                                                                     float cwt_min, uint8_t* __restrict__ code_out,
                                                                     uint32_t* __restrict__ seed_bits, int* status) {
    constexpr int R = kParR;
    __shared__ float ring[kParWarps][kParStages * (kParR + 2) * 32];
    const int N = ng;
    const int nbx = (N + 29) / 30, nby = (N + R - 1) / R;
    const int64_t warp = (int64_t(blockIdx.x) * kParThreads + threadIdx.x) >> 5;
    const int64_t nwarps = int64_t(nbx) * nby * ((N + kParZ - 1) / kParZ);
    if (warp >= nwarps) return;  // warp-uniform
    const int by = int(warp % nby), bx = int((warp / nby) % nbx), bz = int(warp / (int64_t(nby) * nbx));
    const int x0 = bx * 30, y0 = by * R, z0 = bz * kParZ;
    const int wzc = min(kParZ, N - z0);
    float* my_ring = ring[threadIdx.x >> 5];
    // warp-uniform: owned columns x0 .. x0+29 and rows y0 .. y0+R-1 clear of 0 and N-1
    if (x0 > 0 && x0 + 30 < N && y0 > 0 && y0 + R < N)
        parent_block<true, true>(C, N, cwt_min, code_out, seed_bits, status, x0, y0, z0, wzc, my_ring);
    else
        parent_block<false, false>(C, N, cwt_min, code_out, seed_bits, status, x0, y0, z0, wzc, my_ring);
}

// In-tile chains of a 64 x 16 x 16-cell tile from the parent codes.  Every
// cell's code becomes a shared-memory pointer (a local index, a seed's own
// index, -1 for a maximum that is not a seed, or -2 - g for a parent g outside
// the tile); pointer-jumping rounds over the whole tile then bring every
// pointer to the end of its chain inside the tile: a seed, a non-seed maximum,
// or a cell outside the tile.  A cell whose chain ends at a seed of this tile
// adds one to the seed's cell count, kept in the upper half of the seed's own
// entry.
__global__ void __launch_bounds__(kChThreads, 3) k_seg_chase(const uint8_t* __restrict__ codes, int ng,
                                                           int32_t* __restrict__ label,
                                                           uint32_t* __restrict__ seed_cells,
                                                           uint32_t* __restrict__ ballots, int* status) {
    extern __shared__ __align__(16) int32_t ptr[];  // [kLocal], dynamic
    __shared__ uint16_t tile_seeds[kTileSeedCap];
    __shared__ uint32_t n_tile_seeds;
    const int N = ng;  // even
    const int ntx = (N + kChTX - 1) / kChTX, nty = (N + kChTY - 1) / kChTY;
    const int t = int(blockIdx.x);
    const int tx = t % ntx, ty = (t / ntx) % nty, tz = t / (ntx * nty);
    const int x0 = tx * kChTX, y0 = ty * kChTY, z0 = tz * kChTZ;
    const int wx = min(kChTX, N - x0), wy = min(kChTY, N - y0), wz = min(kChTZ, N - z0);  // wx even
    const int lane = threadIdx.x & 31, ly = threadIdx.x >> 5;
    const int lx = 2 * lane;  // this lane's columns lx, lx + 1
    const bool own = lx < wx && ly < wy;
    const int xc = x0 + lx, yc = y0 + ly;
    const int32_t plane32 = N * N;
    // global index pieces of the neighbours (one step, or across the periodic
    // boundary) of the even column xc and the odd column xc + 1
    const int32_t oxm0 = xc == 0 ? N - 1 : -1, oxp1 = xc + 1 == N - 1 ? -(N - 1) : 1;
    const int32_t oym = yc == 0 ? (N - 1) * N : -N, oyp = yc == N - 1 ? -(N - 1) * N : N;
    if (threadIdx.x == 0) n_tile_seeds = 0;
    __syncthreads();
    const int i0 = ly * kPX + lx;
    // a cell's shared-memory pointer from its parent code: a seed's own index,
    // -1 for a maximum that is not a seed, a local index, or -2 - g for a
    // parent g outside the tile
    auto decode = [&](uint32_t code, int cx, int lz, int zc, int32_t g, int32_t oxm, int32_t oxp, int i) -> int32_t {
        if ((code & 0x3fu) == kCodeMax) {
            if (code & kCodeSeed) {
                const uint32_t j = atomicAdd(&n_tile_seeds, 1u);
                if (j < uint32_t(kTileSeedCap)) tile_seeds[j] = uint16_t(i);
                return i;
            }
            return -1;
        }
        const int dx = int(code & 3u) - 1, dy = int((code >> 2) & 3u) - 1, dz = int((code >> 4) & 3u) - 1;
        if (unsigned(cx + dx) < unsigned(wx) && unsigned(ly + dy) < unsigned(wy) && unsigned(lz + dz) < unsigned(wz))
            return i + dx + dy * kPX + dz * kPlaneL;
        const int32_t ozm = zc == 0 ? (N - 1) * plane32 : -plane32;
        const int32_t ozp = zc == N - 1 ? -(N - 1) * plane32 : plane32;
        return -2 - (g + (dx < 0 ? oxm : (dx > 0 ? oxp : 0)) + (dy < 0 ? oym : (dy > 0 ? oyp : 0)) +
                     (dz < 0 ? ozm : (dz > 0 ? ozp : 0)));
    };
    if (own) {
        const int32_t grow = yc * N + xc;  // even
        constexpr int kBatch = 8;  // planes whose codes are loaded together (independent loads in flight)
        for (int lb = 0; lb < wz; lb += kBatch) {
            uint32_t cb[kBatch];
#pragma unroll
            for (int u = 0; u < kBatch; u++)
                cb[u] = lb + u < wz ? *reinterpret_cast<const uint16_t*>(codes + (z0 + lb + u) * plane32 + grow) : 0u;
#pragma unroll
            for (int u = 0; u < kBatch; u++) {
                const int lz = lb + u;
                if (lz >= wz) break;
                const int zc = z0 + lz;
                const int32_t g = zc * plane32 + grow;
                const int i = i0 + lz * kPlaneL;
                int2 v;
                v.x = decode(cb[u] & 0xffu, lx, lz, zc, g, oxm0, 1, i);
                v.y = decode(cb[u] >> 8, lx + 1, lz, zc, g + 1, -1, oxp1, i + 1);
                *reinterpret_cast<int2*>(&ptr[i]) = v;
            }
        }
    }
    __syncthreads();
    // Pointer jumping in place, every cell of the tile in lockstep (no divergent
    // walks): a pointer to a non-root cell moves two links further (the target's
    // target's pointer, so a round triples the distance covered), until no
    // pointer changes.  A value read while another thread rewrites it is either
    // the old or the new pointer, both points of the same chain.
    auto jump1 = [&](int i, int32_t v, bool& changed) {
        if (v >= 0 && v != i && index_ok(v, kLocal, status)) {
            int32_t w = ptr[v];
            if (w != v) {
                if (w >= 0 && index_ok(w, kLocal, status)) w = ptr[w];
                ptr[i] = w;
                changed = true;
            }
        }
    };
    auto jump = [&](int lz, bool& changed) {
        const int i = i0 + lz * kPlaneL;
        const int2 v = *reinterpret_cast<const int2*>(&ptr[i]);
        jump1(i, v.x, changed);
        jump1(i + 1, v.y, changed);
    };
    for (int round = 0; round < kJumpRoundsInTile; round++) {
        bool changed = false;
        if (own) {
            if (wz == kChTZ) {  // every tile but a ragged last one along z
#pragma unroll 8
                for (int lz = 0; lz < kChTZ; lz++) jump(lz, changed);
            } else {
                for (int lz = 0; lz < wz; lz++) jump(lz, changed);
            }
        }
        if (!__syncthreads_or(changed)) break;
    }
    // every pointer now names a root (its cell's seed), -1, or -2 - g (a cell
    // outside): labels, and one count per cell for the tile's seeds, kept in
    // the upper half of the seed's own entry (readers mask it off)
    const int32_t gbase = (z0 * N + y0) * N + x0;
    const unsigned full = 0xffffffffu;
    auto finish = [&](int32_t v, bool& fl) -> int32_t {
        const int32_t cur = v >= 0 ? (v & kLocalMask) : v;
        if (cur == -1) return -1;
        if (cur <= -2) {
            fl = true;
            return cur;  // -2 - g: already the flagged pointer to the outside parent g
        }
        if (!index_ok(cur, kLocal, status)) return -1;
        const int px = cur & (kPX - 1), py = (cur >> kPXBits) & (kChTY - 1), pz = cur >> kPlaneBits;
        const int32_t g = gbase + (pz * N + py) * N + px;
        const int32_t nv = ptr[cur];
        if (nv >= 0 && (nv & kLocalMask) == cur) {
            atomicAdd(&ptr[cur], 1 << kCountShift);
            return g;
        }
        fl = true;
        return -2 - g;  // not finished within the round bound: resume globally
    };
    int32_t* out = label + (size_t(z0) * N + yc) * N + xc;
    const bool vec = (reinterpret_cast<uintptr_t>(label) & 7u) == 0;  // xc is even: 8-byte label pairs
    uint32_t* my_ballots = ballots + (size_t(t) * kChTY + ly) * kRowWords;
    for (int lz = 0; lz < kChTZ; lz++, out += size_t(plane32)) {  // block-uniform trip count
        bool f0 = false, f1 = false;
        if (own && lz < wz) {
            const int i = i0 + lz * kPlaneL;
            const int2 v = *reinterpret_cast<const int2*>(&ptr[i]);
            int2 res;
            res.x = finish(v.x, f0);
            res.y = finish(v.y, f1);
            if (vec) {
                *reinterpret_cast<int2*>(out) = res;
            } else {
                out[0] = res.x;
                out[1] = res.y;
            }
        }
        const unsigned b0 = __ballot_sync(full, f0), b1 = __ballot_sync(full, f1);
        if (lane == 2 * lz) my_ballots[2 * lz] = b0;  // plane lz, even columns
        if (lane == 2 * lz + 1) my_ballots[2 * lz + 1] = b1;  // odd columns
    }
    __syncthreads();
    // in-tile cell counts of this tile's seeds (cells reaching them from other
    // tiles are added by the global pass)
    const uint32_t nts = n_tile_seeds;
    if (threadIdx.x == 0 && nts > uint32_t(kTileSeedCap)) set_status(status, CWTHF_E_BAD_INPUT);
    for (uint32_t j = threadIdx.x; j < min(nts, uint32_t(kTileSeedCap)); j += blockDim.x) {
        const int i = tile_seeds[j];
        const int px = i & (kPX - 1), py = (i >> kPXBits) & (kChTY - 1), pz = i >> kPlaneBits;
        seed_cells[size_t(gbase + (pz * N + py) * N + px)] = uint32_t(ptr[i]) >> kCountShift;
    }
}

constexpr int kResolveThreads = 256;
constexpr int kResTabBits = 9, kResTab = 1 << kResTabBits;  // per-tile count table (shared memory)

// The global pass over the cells whose chain left their tile.  A CTA takes one
// chain tile at a time from a global counter, and its warps take the tile's
// rows one at a time from a shared counter (the flagged cells crowd where the
// field is clumped, so a fixed split leaves some warps far more work than
// others).  A warp gathers the flagged cells of a row's non-empty plane masks
// into a shared batch; every full batch of 32 cells (and the warp's last,
// partial one of the tile) is resolved by the whole warp: each lane follows
// its cell's chain through the label grid (at most `limit` steps, kDefaultChaseLimit
// by default) and takes the label it reaches.  The tile's cells are counted
// per seed in a shared table (one entry per distinct seed, one shared atomic
// per distinct seed of a batch) that is added to the counts kept at the seeds'
// cells once per tile (the tile pass wrote each seed's in-tile count there;
// seed slots are ranked only afterwards).  A cell still unfinished at the
// limit stays flagged and sets changed[0]; the doubling rounds then finish it
// and the cells are recounted.  Labels read while other threads update them
// are always a later point of the same chain, so the result does not depend
// on timing.
__device__ __forceinline__ void table_add(int32_t* tkey, uint32_t* tcnt, uint32_t* __restrict__ seed_cells,
                                          int32_t lab, uint32_t n) {
    uint32_t h = (uint32_t(lab) * 2654435761u) >> (32 - kResTabBits);
    for (int p = 0; p < 16; p++) {
        const int32_t k = tkey[h];
        if (k == lab) {
            atomicAdd(&tcnt[h], n);
            return;
        }
        if (k == -1) {
            const int32_t prev = atomicCAS(&tkey[h], -1, lab);
            if (prev == -1 || prev == lab) {
                atomicAdd(&tcnt[h], n);
                return;
            }
        }
        h = (h + 1) & (kResTab - 1);
    }
    atomicAdd(&seed_cells[lab], n);  // table crowded: straight to the seed's count
}

__device__ __forceinline__ void resolve_batch(int32_t* __restrict__ label, bool valid, uint32_t c, int32_t* tkey,
                                              uint32_t* tcnt, uint32_t* __restrict__ seed_cells, int limit,
                                              bool& left, int64_t cells, int* status) {
    int32_t lab = -1;
    if (valid) {
        int32_t w = label[c];
        int steps = 0;
        while (is_flagged(w) && steps < limit) {
            if (!index_ok(flag_target(w), cells, status)) {
                w = -1;
                break;
            }
            w = label[flag_target(w)];
            steps++;
        }
        label[c] = w;
        if (is_flagged(w)) left = true;
        else lab = w;
    }
    const unsigned peers = __match_any_sync(0xffffffffu, lab);  // every lane
    if (lab >= 0 && (threadIdx.x & 31) == __ffs(peers) - 1)
        table_add(tkey, tcnt, seed_cells, lab, uint32_t(__popc(peers)));
}

__global__ void __launch_bounds__(kResolveThreads) k_seg_resolve(int32_t* __restrict__ label, int ng,
                                                                 const uint32_t* __restrict__ ballots,
                                                                 uint32_t* __restrict__ seed_cells,
                                                                 int* __restrict__ changed,
                                                                 unsigned* __restrict__ next_tile, int limit,
                                                                 int* status) {
    __shared__ uint32_t batch[kResolveThreads / 32][64];  // pending cells (fewer than 32 between batches)
    __shared__ int32_t tkey[kResTab];
    __shared__ uint32_t tcnt[kResTab];
    __shared__ unsigned s_tile, s_row;
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    uint32_t* wl = batch[threadIdx.x >> 5];
    const int N = ng;
    const int ntx = (N + kChTX - 1) / kChTX, nty = (N + kChTY - 1) / kChTY, ntz = (N + kChTZ - 1) / kChTZ;
    const unsigned ntiles = unsigned(ntx) * unsigned(nty) * unsigned(ntz);
    const uint32_t plane32 = uint32_t(N) * uint32_t(N);
    const int64_t cells = int64_t(plane32) * N;
    for (int i = threadIdx.x; i < kResTab; i += blockDim.x) {
        tkey[i] = -1;
        tcnt[i] = 0;
    }
    bool left = false;
    for (;;) {
        if (threadIdx.x == 0) {
            s_tile = atomicAdd(next_tile, 1u);
            s_row = 0;
        }
        __syncthreads();
        const unsigned t = s_tile;
        if (t >= ntiles) break;  // block-uniform
        const int tx = int(t % unsigned(ntx)), ty = int((t / unsigned(ntx)) % unsigned(nty)),
                  tz = int(t / (unsigned(ntx) * unsigned(nty)));
        uint32_t k = 0;  // warp-uniform
        for (;;) {
            unsigned ly = 0;
            if (lane == 0) ly = atomicAdd(&s_row, 1u);
            ly = __shfl_sync(full, ly, 0);
            if (ly >= unsigned(kChTY)) break;  // warp-uniform
            const int yc = ty * kChTY + int(ly);
            if (yc >= N) continue;  // warp-uniform
            const int64_t rw = int64_t(t) * kChTY + ly;
            const uint32_t mine = ballots[rw * kRowWords + lane];  // plane lane / 2, columns of parity lane % 2
            uint32_t words = __ballot_sync(full, mine != 0u);
            const uint32_t cell0 =
                uint32_t((int64_t(tz) * kChTZ * N + yc) * N + int64_t(tx) * kChTX) + 2u * uint32_t(lane);
            while (words) {
                const int wd = __ffs(words) - 1;
                words &= words - 1u;
                const uint32_t b = __shfl_sync(full, mine, wd);
                if (b & (1u << lane)) wl[k + __popc(b & lt)] = cell0 + uint32_t(wd >> 1) * plane32 + uint32_t(wd & 1);
                k += __popc(b);
                if (k >= 32) {
                    __syncwarp();
                    resolve_batch(label, true, wl[lane], tkey, tcnt, seed_cells, limit, left, cells, status);
                    const uint32_t rest = wl[32 + lane];
                    __syncwarp();
                    if (uint32_t(lane) + 32 < k) wl[lane] = rest;
                    k -= 32;
                    __syncwarp();
                }
            }
        }
        __syncwarp();
        if (k)
            resolve_batch(label, uint32_t(lane) < k, uint32_t(lane) < k ? wl[lane] : 0u, tkey, tcnt, seed_cells,
                          limit, left, cells, status);
        __syncthreads();
        // the tile's counts go to the seeds' cells; the table is cleared for the next tile
        for (int i = threadIdx.x; i < kResTab; i += blockDim.x) {
            const int32_t key = tkey[i];
            if (key >= 0) {
                atomicAdd(&seed_cells[key], tcnt[i]);
                tkey[i] = -1;
                tcnt[i] = 0;
            }
        }
        __syncthreads();
    }
    if (__any_sync(full, left) && lane == 0) changed[0] = 1;
}

// Fallback for chains that outlived the bounded walks (changed[0] set by the
// resolve pass); returns at once otherwise.  Round r (1 <= r <= rounds)
// replaces every flagged pointer by its target's label, which moves it 2^(r-1)
// or more links further, so 31 rounds finish any chain of a grid of at most
// 2^30 cells; changed[r] records whether a pointer is still flagged after it.
// Rounds are separated by grid barriers.  Then the cell counts of every seed
// (kept at the seed's cell) are cleared and recounted from the finished
// labels.  A flag still set after
// the last round is reported as CWTHF_E_NOT_CONVERGED (the labels are then
// unspecified, and flagged values are skipped by the recount).
__global__ void __launch_bounds__(256) k_seg_fallback(int32_t* __restrict__ label, int64_t cells, int* changed,
                                                      int rounds, const uint32_t* __restrict__ bits,
                                                      uint32_t* __restrict__ seed_cells, unsigned* bar, int* status) {
    if (*reinterpret_cast<volatile int*>(&changed[0]) == 0) return;  // the same answer in every CTA
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    const int64_t gid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    bool done = false;
    for (int r = 1; r <= rounds; r++) {
        bool any = false;
        for (int64_t c = gid; c < cells; c += stride) {
            const int32_t v = label[c];
            if (is_flagged(v) && index_ok(flag_target(v), cells, status)) {
                const int32_t w = label[flag_target(v)];
                label[c] = w;
                any |= is_flagged(w);  // still a pointer: another round is needed
            }
        }
        if (__any_sync(0xffffffffu, any) && (threadIdx.x & 31) == 0) atomicOr(&changed[r], 1);
        if (!grid_sync(bar, status)) return;
        if (*reinterpret_cast<volatile int*>(&changed[r]) == 0) {
            done = true;
            break;
        }
    }
    if (!done && gid == 0) set_status(status, CWTHF_E_NOT_CONVERGED);
    auto is_seed = [&](int64_t c) { return (bits[c >> 5] >> (c & 31)) & 1u; };
    for (int64_t c = gid; c < cells; c += stride)
        if (is_seed(c)) seed_cells[c] = 0;
    if (!grid_sync(bar, status)) return;
    for (int64_t c = gid; c < cells; c += stride) {
        const int32_t l = label[c];
        if (l >= 0 && int64_t(l) < cells && is_seed(l)) atomicAdd(&seed_cells[l], 1u);
    }
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
                            int64_t slot_cap, int32_t* __restrict__ seed_list, const uint32_t* __restrict__ seed_cells,
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

// Seeds of the last segmentation and their segments' cell counts.
__global__ void k_segment_sizes(const int32_t* __restrict__ seed_list, const HaloAcc* __restrict__ acc,
                                const uint32_t* __restrict__ n_slots, int64_t cap, int32_t* __restrict__ seeds,
                                int64_t* __restrict__ n_cells, int64_t* __restrict__ n_out) {
    const int64_t ns = *n_slots;
    if (blockIdx.x == 0 && threadIdx.x == 0) *n_out = ns;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < min(ns, cap); i += stride) {
        seeds[i] = seed_list[i];
        n_cells[i] = int64_t(acc[i].n_cells);
    }
}

}  // namespace

int segment_sizes_impl(cwthf_ctx* ctx, int32_t* seeds, int64_t* n_cells, int64_t cap, int64_t* n_seeds,
                       cudaStream_t s) {
    CWTHF_LAUNCH(ctx, s, "k_segment_sizes",
                 k_segment_sizes<<<ctx->sm_count, 256, 0, s>>>(ctx->seed_list, ctx->acc, ctx->n_seeds, cap, seeds,
                                                               n_cells, n_seeds));
    return cuda_status(cudaGetLastError());
}

int seeds_rank(cwthf_ctx* ctx, int ng, const uint32_t* seed_cells, cudaStream_t s) {
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

// CTAs of the cooperative fallback launch: all resident at once (its grid
// barriers need that), at most four per SM.
int fallback_blocks(int sm_count) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_seg_fallback, 256, 0) != cudaSuccess || per_sm < 1)
        return -1;
    return std::min(per_sm, 4) * sm_count;
}

int launch_fallback(cwthf_ctx* ctx, int32_t* label, int64_t cells, cudaStream_t s) {
    if (ctx->fallback_blocks <= 0) return CWTHF_E_CUDA;
    int* changed = ctx->jump_changed;
    unsigned* bar = reinterpret_cast<unsigned*>(changed + kJumpBarrier);
    int rounds = ctx->dbg_jump_rounds;
    void* args[] = {&label, &cells, &changed, &rounds, &ctx->seed_bits, &ctx->seed_cells, &bar, &ctx->d_status};
    cudaError_t e;
    CWTHF_LAUNCH(ctx, s, "k_seg_fallback",
                 e = cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(&k_seg_fallback),
                                                 dim3(unsigned(ctx->fallback_blocks)), dim3(256), args, 0, s));
    return cuda_status(e);
}

int segment_impl(cwthf_ctx* ctx, const float* cwt, int ng, float cwt_min, int32_t* label, bool,
                 cudaStream_t s) {
    int64_t cells = int64_t(ng) * ng * ng;
    int64_t nwords = (cells + 31) / 32;
    cudaError_t e = cudaMemsetAsync(ctx->seed_bits, 0, size_t(nwords) * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->jump_changed, 0, sizeof(int) * kJumpWords, s);
    if (e != cudaSuccess) return cuda_status(e);
    // parent codes (1 byte per cell) and the flagged-cell masks of every chain
    // tile (one bit per cell) in the context's int64 grid buffer (8 bytes per
    // cell, free once the forward transform has read it), then the in-tile chains
    uint8_t* codes = reinterpret_cast<uint8_t*>(ctx->grid);
    uint32_t* ballots = reinterpret_cast<uint32_t*>(codes + (size_t(cells) + 255) / 256 * 256);
    const int64_t ntiles = int64_t(div_up(ng, kChTX)) * div_up(ng, kChTY) * div_up(ng, kChTZ);
    if ((cells + 255) / 256 * 256 + ntiles * (kChTY * kRowWords * 4) > cells * 8) return CWTHF_E_UNSUPPORTED_SIZE;
    const int64_t pwarps = int64_t(div_up(ng, 30)) * div_up(ng, kParR) * div_up(ng, kParZ);
    CWTHF_LAUNCH(ctx, s, "k_seg_parent",
                 k_seg_parent<<<unsigned(div_up(pwarps, int64_t(kParWarps))), kParThreads, 0, s>>>(
                     cwt, ng, cwt_min, codes, ctx->seed_bits, ctx->d_status));
    cudaFuncSetAttribute(k_seg_chase, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sizeof(int32_t) * kLocal));
    CWTHF_LAUNCH(ctx, s, "k_seg_chase",
                 k_seg_chase<<<unsigned(ntiles), kChThreads, sizeof(int32_t) * kLocal, s>>>(
                     codes, ng, label, ctx->seed_cells, ballots, ctx->d_status));
    // chains that left their tile, counted at their seed's cell
    int blocks = ctx->sm_count * 8;
    int* changed = ctx->jump_changed;  // see kJumpWords
    CWTHF_LAUNCH(ctx, s, "k_seg_resolve",
                 k_seg_resolve<<<blocks, kResolveThreads, 0, s>>>(label, ng, ballots, ctx->seed_cells, changed,
                                                                   reinterpret_cast<unsigned*>(changed + kJumpTileCounter),
                                                                   ctx->dbg_chase_limit, ctx->d_status));
    // pointer doubling and a recount for whatever the bounded walks left
    // (normally nothing: the kernel then returns at once)
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e);
    int rc = launch_fallback(ctx, label, cells, s);
    if (rc) return rc;
    // seed slots in cell order, each with its segment's cell count
    return seeds_rank(ctx, ng, ctx->seed_cells, s);
}

}  // namespace cwthf
