// stencil.cu -- the grid CWT as the paper evaluates it (Sec. 2.1): every grid
// node adds its mass times the wavelet sampled on a stencil around it.  The
// stencil is the cube of offsets |d_x|, |d_y|, |d_z| <= R (R = gdw_resolution
// of Table 1, read as a radius), periodic:
//   C(g) = sum_{d in cube} m(g - d) Psi(w, Delta |d|).
//
// On a cube the Mexican hat stays exactly separable: with G(d) = exp(-w^2
// Delta^2 d^2 / 4) and H(d) = w^2 Delta^2 d^2 G(d) (both even, |d| <= R),
//   Psi = w^1.5 [6 G_x G_y G_z - H_x G_y G_z - G_x H_y G_z - G_x G_y H_z],
// so the sum is seven 1D convolutions in three passes over the grid:
//   x:  A = G_x * m,  B = H_x * m
//   y:  P = G_y * (6A - B) - H_y * A,  Q = G_y * A
//   z:  C = w^1.5 (G_z * P - H_z * Q).
// Each pass reads and writes the grid once (8 + 8, 8 + 8, 8 + 4 bytes per
// cell), in fp32, with the int64 CIC masses converted on the first read.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.cuh"

namespace cwthf {
namespace {

constexpr int kMaxR = CWTHF_MAX_STENCIL_R;

struct StencilTaps {
    float g[kMaxR + 1];  // G(d), d = 0..R
    float h[kMaxR + 1];  // H(d)
    int R;
};

constexpr int kXWarps = 8;  // rows per CTA in the x pass

// x pass: one warp per row of the grid.  The row (with R wrapped cells on each
// side) is staged in shared memory; each lane then forms A and B for the
// columns lane, lane + 32, ...
__global__ void __launch_bounds__(32 * kXWarps) k_sten_x(const int64_t* __restrict__ grid, int ng, StencilTaps t,
                                                         float* __restrict__ A, float* __restrict__ B) {
    extern __shared__ float rows[];  // [kXWarps][ng + 2R]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int R = t.R, W = ng + 2 * R;
    float* buf = rows + warp * W;
    const int64_t nrows = int64_t(ng) * ng;
    const int64_t row = int64_t(blockIdx.x) * kXWarps + warp;
    if (row >= nrows) return;  // warp-uniform; no block barrier below
    constexpr float kUnit = 9.3132257461547852e-10f;  // 2^-30: one CIC mass unit
    const int64_t* src = grid + row * ng;
    for (int j = lane; j < W; j += 32) {
        int x = j - R;
        x = x < 0 ? x + ng : (x >= ng ? x - ng : x);
        buf[j] = __ll2float_rn(src[x]) * kUnit;
    }
    __syncwarp();
    float* a = A + row * ng;
    float* b = B + row * ng;
    for (int x = lane; x < ng; x += 32) {
        const float* c = buf + x + R;  // c[d] = m(x + d)
        float sa = t.g[0] * c[0], sb = 0.0f;  // H(0) = 0
        for (int d = 1; d <= R; d++) {
            const float s = c[-d] + c[d];
            sa = fmaf(t.g[d], s, sa);
            sb = fmaf(t.h[d], s, sb);
        }
        a[x] = sa;
        b[x] = sb;
    }
}

// y and z passes: a CTA takes 32 adjacent x columns of one line family (a
// plane z for the y pass, a row y for the z pass) and kLine outputs along the
// pass's axis, staging kLine + 2R input lines of both arrays in shared memory.
constexpr int kLine = 64;
constexpr int kLineThreads = 256;

template <bool kZ>
__global__ void __launch_bounds__(kLineThreads) k_sten_yz(const float* __restrict__ in0, const float* __restrict__ in1,
                                                         int ng, StencilTaps t, float scale,
                                                         float* __restrict__ out0, float* __restrict__ out1) {
    extern __shared__ float tile[];  // [2][kLine + 2R][32]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int R = t.R, H = kLine + 2 * R;
    float* s0 = tile;
    float* s1 = tile + H * 32;
    const int nxc = (ng + 31) / 32, nlc = (ng + kLine - 1) / kLine;
    const int xc = int(blockIdx.x % nxc), lc = int((blockIdx.x / nxc) % nlc), fam = int(blockIdx.x / (nxc * nlc));
    const int x = xc * 32 + lane;
    const bool own = x < ng;
    const int64_t stride = kZ ? int64_t(ng) * ng : int64_t(ng);  // step along the pass's axis
    const int64_t base = (kZ ? int64_t(fam) * ng : int64_t(fam) * ng * ng) + x;
    const int l0 = lc * kLine;
    for (int j = warp; j < H; j += kLineThreads / 32) {
        int l = l0 - R + j;
        l = ((l % ng) + ng) % ng;
        float v0 = 0.f, v1 = 0.f;
        if (own) {
            v0 = in0[base + l * stride];
            v1 = in1[base + l * stride];
        }
        if (kZ) {  // z pass: inputs P, Q as they are
            s0[j * 32 + lane] = v0;
            s1[j * 32 + lane] = v1;
        } else {  // y pass: inputs A, B; stage U = 6A - B and A
            s0[j * 32 + lane] = 6.0f * v0 - v1;
            s1[j * 32 + lane] = v0;
        }
    }
    __syncthreads();
    if (!own) return;
    for (int j = warp; j < kLine; j += kLineThreads / 32) {
        const int l = l0 + j;
        if (l >= ng) break;
        const float* c0 = s0 + (j + R) * 32 + lane;
        const float* c1 = s1 + (j + R) * 32 + lane;
        if (kZ) {  // C = scale (G * P - H * Q)
            float sp = t.g[0] * c0[0], sq = 0.0f;
            for (int d = 1; d <= R; d++) {
                sp = fmaf(t.g[d], c0[-32 * d] + c0[32 * d], sp);
                sq = fmaf(t.h[d], c1[-32 * d] + c1[32 * d], sq);
            }
            out0[base + l * stride] = scale * (sp - sq);
        } else {  // P = G * U - H * A,  Q = G * A
            float su = t.g[0] * c0[0], sa = t.g[0] * c1[0], sh = 0.0f;
            for (int d = 1; d <= R; d++) {
                const float a = c1[-32 * d] + c1[32 * d];
                su = fmaf(t.g[d], c0[-32 * d] + c0[32 * d], su);
                sa = fmaf(t.g[d], a, sa);
                sh = fmaf(t.h[d], a, sh);
            }
            out0[base + l * stride] = su - sh;
            out1[base + l * stride] = sa;
        }
    }
}

}  // namespace

int transform_stencil_impl(cwthf_ctx* ctx, const int64_t* grid, int ng, double L, double mass_unit, double w, int R,
                           float* cwt, cudaStream_t s) {
    StencilTaps t;
    t.R = R;
    const double dx = L / ng;
    for (int d = 0; d <= R; d++) {
        const double u2 = (dx * d) * (dx * d);
        const double gd = std::exp(-0.25 * w * w * u2);
        t.g[d] = float(gd);
        t.h[d] = float(w * w * u2 * gd);
    }
    const float scale = float(std::pow(w, 1.5) * mass_unit);
    const int64_t cells = int64_t(ng) * ng * ng;
    // scratch: A, B in the context's CWT and label buffers, P, Q in its int64
    // grid buffer (two float grids)
    float* A = ctx->cwt;
    float* B = reinterpret_cast<float*>(ctx->label);
    float* P = reinterpret_cast<float*>(ctx->grid);
    float* Q = P + cells;
    const size_t xs = size_t(kXWarps) * (ng + 2 * R) * sizeof(float);
    const int xblocks = div_up(int64_t(ng) * ng, kXWarps);
    CWTHF_LAUNCH(ctx, s, "k_sten_x", k_sten_x<<<xblocks, 32 * kXWarps, xs, s>>>(grid, ng, t, A, B));
    const size_t ls = size_t(2) * (kLine + 2 * R) * 32 * sizeof(float);
    const unsigned lblocks = unsigned(div_up(ng, 32) * div_up(ng, kLine) * ng);
    cudaFuncSetAttribute(k_sten_yz<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(ls));
    cudaFuncSetAttribute(k_sten_yz<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(ls));
    CWTHF_LAUNCH(ctx, s, "k_sten_y", k_sten_yz<false><<<lblocks, kLineThreads, ls, s>>>(A, B, ng, t, 1.0f, P, Q));
    CWTHF_LAUNCH(ctx, s, "k_sten_z", k_sten_yz<true><<<lblocks, kLineThreads, ls, s>>>(P, Q, ng, t, scale, cwt, nullptr));
    return cuda_status(cudaGetLastError());
}

}  // namespace cwthf
