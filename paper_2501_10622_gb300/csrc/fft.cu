// fft.cu -- the grid CWT of Sec. 2.1 (Eq. 2-4) as a 3D real FFT, a multiply
// by the exact DFT of the sampled Mexican-hat wavelet, and an inverse FFT.
//
// Data flow for an ng^3 grid (M = ng/2, P = complex row pitch, even):
//   x-fwd   int64 grid -> fp32 -> real FFT along x -> spec [z][y][0..M]   (k_fft_x_fwd)
//   y-fwd   complex FFT along y, in place                                (k_fft_yz, TMA)
//   z       complex FFT along z, multiply by Psi^, inverse FFT along z    (k_fft_yz, TMA)
//   y-inv   inverse complex FFT along y, in place                        (k_fft_yz, TMA)
//   x-inv   half spectrum -> real row, written to the CWT field          (k_fft_x_inv)
//
// Every 1D transform of length L runs in shared memory as a Stockham
// autosort FFT with at most three radix stages (radices 2^a 3^b 5^c 7^d
// <= 32); each
// thread performs one radix-R butterfly per stage entirely in registers, with
// compile-time constants inside the butterfly and fp32 twiddles (rounded once
// from fp64 on the host) between stages.  Inverse transforms use
// IDFT(x) = conj(DFT(conj(x))).  The forward transform is unnormalised; the
// 1/ng^3 of the inverse is folded into the wavelet spectrum.
//
// Wavelet spectrum (exact DFT of the sampled kernel): with G(u) =
// exp(-w^2 u^2/4) and H(u) = w^2 u^2 G(u) sampled at minimum-image offsets,
//   Psi = w^1.5 [6 G_x G_y G_z - H_x G_y G_z - G_x H_y G_z - G_x G_y H_z],
// so its DFT is the same combination of the 1D DFTs G^ and H^ (real, even),
// tabulated per grid size and scale in fp64 on the host.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>

#include "internal.cuh"

namespace cwthf {

struct Tables {
    int ng = 0;
    const float2* twN = nullptr;  // [ng]   exp(-2 pi i m / ng)
    const float2* twM = nullptr;  // [ng/2] exp(-2 pi i m / (ng/2))
    // Bluestein passes (null for passes with a radix plan): chirp b_n of the
    // pass length, the transformed chirp of the inner length (scaled by its
    // inverse), the inner length's twiddles
    const float2* chirp_yz = nullptr;
    const float2* bhat_yz = nullptr;
    const float2* tw_yz = nullptr;
    const float2* chirp_x = nullptr;
    const float2* bhat_x = nullptr;
    const float2* tw_x = nullptr;
};

namespace {

// ---------------------------------------------------------------------------
// Compile-time twiddle constants (series evaluated in fp64, rounded to fp32).
// ---------------------------------------------------------------------------
constexpr double kPi = 3.14159265358979323846264338327950288;

__host__ __device__ constexpr double cx_sin(double x) {
    double term = x, sum = x;
    for (int k = 1; k < 30; k++) {
        term *= -x * x / double((2 * k) * (2 * k + 1));
        sum += term;
    }
    return sum;
}
__host__ __device__ constexpr double cx_cos(double x) {
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 30; k++) {
        term *= -x * x / double((2 * k - 1) * (2 * k));
        sum += term;
    }
    return sum;
}
// angle 2 pi e / n reduced into [-pi, pi]
__host__ __device__ constexpr double cx_angle(int e, int n) {
    int r = ((e % n) + n) % n;
    if (2 * r > n) r -= n;
    return 2.0 * kPi * double(r) / double(n);
}

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }

// a * exp(-2 pi i E / N), exact for the quarter turns.
template <int N, int E>
__device__ __forceinline__ float2 mul_w(float2 a) {
    constexpr int e = ((E % N) + N) % N;
    if constexpr (e == 0) {
        return a;
    } else if constexpr (4 * e == N) {
        return make_float2(a.y, -a.x);
    } else if constexpr (2 * e == N) {
        return make_float2(-a.x, -a.y);
    } else if constexpr (4 * e == 3 * N) {
        return make_float2(-a.y, a.x);
    } else {
        constexpr float wr = float(cx_cos(cx_angle(e, N)));
        constexpr float wi = float(-cx_sin(cx_angle(e, N)));
        return make_float2(a.x * wr - a.y * wi, a.x * wi + a.y * wr);
    }
}

template <int I, int End, class F>
__device__ __forceinline__ void static_for(F&& f) {
    if constexpr (I < End) {
        f(std::integral_constant<int, I>{});
        static_for<I + 1, End>(f);
    }
}

// Smallest prime factor of n (2, 3, 5 or 7 for the supported radices).
__host__ __device__ constexpr int small_factor(int n) {
    return n % 2 == 0 ? 2 : (n % 3 == 0 ? 3 : (n % 5 == 0 ? 5 : 7));
}

// Position of output k of the in-place DIF below: for N = p*M, X[p*m + s]
// ends in block s at the position its length-M sub-transform gives m.
__host__ __device__ constexpr int dig_rev(int n, int k) {
    int pos = 0, base = 0;
    while (n > 1) {
        int p = small_factor(n), m = n / p;
        base += m * (k % p);
        k /= p;
        n = m;
    }
    return base + pos;
}

// In-register forward DFT of N values (N = 2^a 3^b 5^c 7^d), decimation in
// frequency, in place on v[OFF .. OFF+N): input in natural order, output
// X[k] at v[OFF + dig_rev(N, k)].  All indices are compile-time constants.
// Each step splits N = P M on the smallest prime P: for k < M the P inputs
// k + p M go through a P-point DFT, output q is multiplied by
// exp(-2 pi i q k / N) and kept in block q, whose length-M DFT follows.
template <int N>
struct RegDif {
    static constexpr int P = small_factor(N);
    static constexpr int M = N / P;
    template <int OFF>
    static __device__ __forceinline__ void run(float2* v) {
        if constexpr (N > 1) {
            if constexpr (P == 2) {
                static_for<0, M>([&](auto kc) {
                    constexpr int k = decltype(kc)::value;
                    float2 a = v[OFF + k], b = v[OFF + k + M];
                    v[OFF + k] = cadd(a, b);
                    v[OFF + k + M] = mul_w<N, k>(csub(a, b));
                });
            } else if constexpr (P == 3) {
                constexpr float h = 0.866025403784438646763723170752936f;  // sqrt(3)/2
                static_for<0, M>([&](auto kc) {
                    constexpr int k = decltype(kc)::value;
                    float2 a = v[OFF + k], b = v[OFF + k + M], c = v[OFF + k + 2 * M];
                    float2 t1 = cadd(b, c);
                    float2 t2 = make_float2(a.x - 0.5f * t1.x, a.y - 0.5f * t1.y);
                    float2 d = make_float2(h * (b.x - c.x), h * (b.y - c.y));
                    v[OFF + k] = cadd(a, t1);
                    v[OFF + k + M] = mul_w<N, k>(make_float2(t2.x + d.y, t2.y - d.x));          // t2 - i d
                    v[OFF + k + 2 * M] = mul_w<N, 2 * k>(make_float2(t2.x - d.y, t2.y + d.x));  // t2 + i d
                });
            } else {  // P = 5 or 7: the P-point DFT with constant roots
                static_for<0, M>([&](auto kc) {
                    constexpr int k = decltype(kc)::value;
                    float2 a[P];
                    static_for<0, P>([&](auto pc) { a[decltype(pc)::value] = v[OFF + k + decltype(pc)::value * M]; });
                    static_for<0, P>([&](auto qc) {
                        constexpr int q = decltype(qc)::value;
                        float2 y = a[0];
                        static_for<1, P>([&](auto pc) {
                            constexpr int pp = decltype(pc)::value;
                            y = cadd(y, mul_w<P, (pp * q) % P>(a[pp]));
                        });
                        v[OFF + k + q * M] = mul_w<N, q * k>(y);
                    });
                });
            }
            static_for<0, P>([&](auto sc) {
                constexpr int sblk = decltype(sc)::value;
                RegDif<M>::template run<OFF + sblk * M>(v);
            });
        }
    }
};

// ---------------------------------------------------------------------------
// Stockham stages over a shared-memory tile holding C sequences of length L.
// Element l of sequence c lives at Addr(l, c).
// ---------------------------------------------------------------------------
struct Plan {
    int L;       // transform length (the inner length Mb of a Bluestein pass)
    int nst;     // number of stages (1..3)
    int rad[3];  // radices, applied in this order (Ns = product of the earlier ones)
    int C;       // sequences per tile
    int T;       // threads per block (multiple of 32)
    int Lb = 0;  // Bluestein pass: the pass length (L >= 2 Lb - 1), else 0
    const float2* chirp = nullptr;  // [Lb] b_n = exp(i pi n^2 / Lb)
    const float2* bhat = nullptr;   // [L]  DFT_L of the wrapped chirp, divided by L
};

struct AddrPlain {  // [L][C], row-major (TMA tiles)
    int C;
    __device__ __forceinline__ int operator()(int l, int c) const { return l * C + c; }
};
struct AddrSwz {  // [L][C] with the column XOR-swizzled by the row (C a power of 2)
    int C;
    __device__ __forceinline__ int operator()(int l, int c) const { return l * C + (c ^ (l & (C - 1))); }
};

// Load the R inputs of butterfly j, apply the inter-stage twiddles, DFT.
template <int R, class A>
__device__ __forceinline__ void bfly_load(const float2* tile, A addr, const float2* tw, int L, int Ns, int j, int c,
                                          float2 (&v)[R]) {
    const int stride = L / R;
#pragma unroll
    for (int r = 0; r < R; r++) v[r] = tile[addr(j + r * stride, c)];
    if (Ns > 1) {
        const int k = j % Ns;
        const int step = L / (Ns * R);
#pragma unroll
        for (int r = 1; r < R; r++) v[r] = cmul(v[r], tw[r * k * step]);  // r*k*step < Ns*R*step = L
    }
    RegDif<R>::template run<0>(v);  // output r now sits at v[dig_rev(R, r)]
}

template <int R, class A>
__device__ __forceinline__ void bfly_store(float2* tile, A addr, int Ns, int j, int c, const float2 (&v)[R]) {
    const int k = j % Ns;
    const int base = (j / Ns) * Ns * R + k;
    static_for<0, R>([&](auto rc) {
        constexpr int r = decltype(rc)::value;
        tile[addr(base + r * Ns, c)] = v[dig_rev(R, r)];
    });
}

// One full stage: every active thread reads, the block syncs, every active thread writes.
// Not inlined: each radix gets its own register allocation.
template <int R, class A>
__device__ __noinline__ void stage_r(float2* tile, A addr, const float2* tw, int L, int Ns, int C) {
    const int c = threadIdx.x % C, j = threadIdx.x / C;
    const bool on = j < L / R;
    float2 v[R];
    if (on) bfly_load<R>(tile, addr, tw, L, Ns, j, c, v);
    __syncthreads();
    if (on) bfly_store<R>(tile, addr, Ns, j, c, v);
    __syncthreads();
}

// The same stage with two butterflies per thread, for tiles whose C L / R
// butterflies exceed the block (up to twice its threads): every thread loads
// both of its butterflies before the barrier and stores them after it, as the
// in-place stage needs.
template <int R, class A>
__device__ __noinline__ void stage_r2(float2* tile, A addr, const float2* tw, int L, int Ns, int C) {
    const int nb = C * (L / R);
    float2 v[2][R];
#pragma unroll
    for (int k = 0; k < 2; k++) {
        const int b = int(threadIdx.x) + k * int(blockDim.x);
        if (b < nb) bfly_load<R>(tile, addr, tw, L, Ns, b / C, b % C, v[k]);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 2; k++) {
        const int b = int(threadIdx.x) + k * int(blockDim.x);
        if (b < nb) bfly_store<R>(tile, addr, Ns, b / C, b % C, v[k]);
    }
    __syncthreads();
}

// A stage of radix R; with kTwo, a stage of radix <= 16 may take two
// butterflies per thread (the plan rule keeps larger radices to one).
template <bool kTwo = false, class A>
__device__ __forceinline__ void stage(int R, float2* tile, A addr, const float2* tw, int L, int Ns, int C) {
    if constexpr (kTwo) {
        if (C * (L / R) > int(blockDim.x)) {
            switch (R) {
                case 2: stage_r2<2>(tile, addr, tw, L, Ns, C); return;
                case 3: stage_r2<3>(tile, addr, tw, L, Ns, C); return;
                case 4: stage_r2<4>(tile, addr, tw, L, Ns, C); return;
                case 5: stage_r2<5>(tile, addr, tw, L, Ns, C); return;
                case 6: stage_r2<6>(tile, addr, tw, L, Ns, C); return;
                case 7: stage_r2<7>(tile, addr, tw, L, Ns, C); return;
                case 8: stage_r2<8>(tile, addr, tw, L, Ns, C); return;
                case 9: stage_r2<9>(tile, addr, tw, L, Ns, C); return;
                case 10: stage_r2<10>(tile, addr, tw, L, Ns, C); return;
                case 12: stage_r2<12>(tile, addr, tw, L, Ns, C); return;
                case 14: stage_r2<14>(tile, addr, tw, L, Ns, C); return;
                case 15: stage_r2<15>(tile, addr, tw, L, Ns, C); return;
                case 16: stage_r2<16>(tile, addr, tw, L, Ns, C); return;
                default: return;
            }
        }
    }
    switch (R) {
        case 2: stage_r<2>(tile, addr, tw, L, Ns, C); break;
        case 3: stage_r<3>(tile, addr, tw, L, Ns, C); break;
        case 4: stage_r<4>(tile, addr, tw, L, Ns, C); break;
        case 5: stage_r<5>(tile, addr, tw, L, Ns, C); break;
        case 6: stage_r<6>(tile, addr, tw, L, Ns, C); break;
        case 7: stage_r<7>(tile, addr, tw, L, Ns, C); break;
        case 8: stage_r<8>(tile, addr, tw, L, Ns, C); break;
        case 9: stage_r<9>(tile, addr, tw, L, Ns, C); break;
        case 10: stage_r<10>(tile, addr, tw, L, Ns, C); break;
        case 12: stage_r<12>(tile, addr, tw, L, Ns, C); break;
        case 14: stage_r<14>(tile, addr, tw, L, Ns, C); break;
        case 15: stage_r<15>(tile, addr, tw, L, Ns, C); break;
        case 16: stage_r<16>(tile, addr, tw, L, Ns, C); break;
        case 18: stage_r<18>(tile, addr, tw, L, Ns, C); break;
        case 20: stage_r<20>(tile, addr, tw, L, Ns, C); break;
        case 21: stage_r<21>(tile, addr, tw, L, Ns, C); break;
        case 24: stage_r<24>(tile, addr, tw, L, Ns, C); break;
        case 25: stage_r<25>(tile, addr, tw, L, Ns, C); break;
        case 27: stage_r<27>(tile, addr, tw, L, Ns, C); break;
        case 28: stage_r<28>(tile, addr, tw, L, Ns, C); break;
        case 30: stage_r<30>(tile, addr, tw, L, Ns, C); break;
        case 32: stage_r<32>(tile, addr, tw, L, Ns, C); break;
        default: break;
    }
}

// Forward DFT of all C sequences of the tile (natural order in and out);
// kTwo: stages may take two butterflies per thread (Bluestein tiles).
template <bool kTwo = false, class A>
__device__ __forceinline__ void fft_tile(const Plan& p, float2* tile, A addr, const float2* tw) {
    const int r0 = p.rad[0], r1 = p.rad[1], r2 = p.rad[2];
    stage<kTwo>(r0, tile, addr, tw, p.L, 1, p.C);
    if (p.nst > 1) stage<kTwo>(r1, tile, addr, tw, p.L, r0, p.C);
    if (p.nst > 2) stage<kTwo>(r2, tile, addr, tw, p.L, r0 * r1, p.C);
}

// Wavelet multiply between the forward and inverse z transforms, done in the
// registers of the last forward stage: the thread that finishes forward
// butterfly j holds X[j + r L/R], exactly the inputs of inverse butterfly j of
// an inverse plan that starts with the same radix R.
struct Wave {
    float a, b;            // this column's coefficients: Psi^(kz) = a G^(kz) + b H^(kz)
    const float* gz;       // G^ table (shared memory)
    const float* hz;       // H^ table (shared memory)
};

template <int R, class A>
__device__ __noinline__ void stage_fused_r(float2* tile, A addr, const float2* tw, int L, int Ns, int C,
                                              const Wave& wv) {
    const int c = threadIdx.x % C, j = threadIdx.x / C;
    const bool on = j < L / R;
    float2 v[R];
    if (on) {
        bfly_load<R>(tile, addr, tw, L, Ns, j, c, v);  // last forward stage: Ns * R == L
        // forward output r (frequency kz = j + r*Ns) sits at v[dig_rev(R, r)]; the first
        // inverse butterfly needs its inputs in natural order r
        float2 u[R];
        static_for<0, R>([&](auto rc) {
            constexpr int r = decltype(rc)::value;
            int kz = j + r * Ns;
            float psi = wv.a * wv.gz[kz] + wv.b * wv.hz[kz];
            float2 x = v[dig_rev(R, r)];
            u[r] = make_float2(x.x * psi, -(x.y * psi));  // multiply, then conj for the inverse
        });
#pragma unroll
        for (int r = 0; r < R; r++) v[r] = u[r];
        RegDif<R>::template run<0>(v);  // first inverse stage (Ns = 1, no twiddles)
    }
    __syncthreads();
    if (on) bfly_store<R>(tile, addr, 1, j, c, v);
    __syncthreads();
}

template <class A>
__device__ __forceinline__ void stage_fused(int R, float2* tile, A addr, const float2* tw, int L, int Ns, int C,
                                            const Wave& wv) {
    switch (R) {
        case 2: stage_fused_r<2>(tile, addr, tw, L, Ns, C, wv); break;
        case 3: stage_fused_r<3>(tile, addr, tw, L, Ns, C, wv); break;
        case 4: stage_fused_r<4>(tile, addr, tw, L, Ns, C, wv); break;
        case 5: stage_fused_r<5>(tile, addr, tw, L, Ns, C, wv); break;
        case 6: stage_fused_r<6>(tile, addr, tw, L, Ns, C, wv); break;
        case 7: stage_fused_r<7>(tile, addr, tw, L, Ns, C, wv); break;
        case 8: stage_fused_r<8>(tile, addr, tw, L, Ns, C, wv); break;
        case 9: stage_fused_r<9>(tile, addr, tw, L, Ns, C, wv); break;
        case 10: stage_fused_r<10>(tile, addr, tw, L, Ns, C, wv); break;
        case 12: stage_fused_r<12>(tile, addr, tw, L, Ns, C, wv); break;
        case 14: stage_fused_r<14>(tile, addr, tw, L, Ns, C, wv); break;
        case 15: stage_fused_r<15>(tile, addr, tw, L, Ns, C, wv); break;
        case 16: stage_fused_r<16>(tile, addr, tw, L, Ns, C, wv); break;
        case 18: stage_fused_r<18>(tile, addr, tw, L, Ns, C, wv); break;
        case 20: stage_fused_r<20>(tile, addr, tw, L, Ns, C, wv); break;
        case 21: stage_fused_r<21>(tile, addr, tw, L, Ns, C, wv); break;
        case 24: stage_fused_r<24>(tile, addr, tw, L, Ns, C, wv); break;
        case 25: stage_fused_r<25>(tile, addr, tw, L, Ns, C, wv); break;
        case 27: stage_fused_r<27>(tile, addr, tw, L, Ns, C, wv); break;
        case 28: stage_fused_r<28>(tile, addr, tw, L, Ns, C, wv); break;
        case 30: stage_fused_r<30>(tile, addr, tw, L, Ns, C, wv); break;
        case 32: stage_fused_r<32>(tile, addr, tw, L, Ns, C, wv); break;
        default: break;
    }
}

// ---------------------------------------------------------------------------
// Compile-time stages for the sizes the large grids use: length, columns and
// radices are constants, so index arithmetic folds to shifts and constants,
// everything inlines into the kernel (one register allocation, no calls), and
// the conjugations of the inverse transforms ride on the first load and the
// last store instead of separate passes over the tile.
// ---------------------------------------------------------------------------
template <int L, int C, int R, int Ns, bool kConjIn, bool kConjOut, class A>
__device__ __forceinline__ void stage_ct(float2* tile, A addr, const float2* tw) {
    constexpr int NB = L / R;  // butterflies per sequence
    const int c = int(threadIdx.x) % C, j = int(threadIdx.x) / C;
    const bool on = j < NB;
    float2 v[R];
    if (on) {
#pragma unroll
        for (int r = 0; r < R; r++) {
            v[r] = tile[addr(j + r * NB, c)];
            if (kConjIn) v[r].y = -v[r].y;
        }
        if constexpr (Ns > 1) {
            const int k = j % Ns;
            constexpr int step = L / (Ns * R);
#pragma unroll
            for (int r = 1; r < R; r++) v[r] = cmul(v[r], tw[r * k * step]);
        }
        RegDif<R>::template run<0>(v);
    }
    __syncthreads();
    if (on) {
        const int k = j % Ns;
        const int base = (j / Ns) * Ns * R + k;
        static_for<0, R>([&](auto rc) {
            constexpr int r = decltype(rc)::value;
            float2 x = v[dig_rev(R, r)];
            if (kConjOut) x.y = -x.y;
            tile[addr(base + r * Ns, c)] = x;
        });
    }
    __syncthreads();
}

// The fused stage of the wavelet transform with constant sizes: last forward
// stage (Ns * R == L), multiply by Psi^ and conjugate, first inverse stage.
template <int L, int C, int R, int Ns, class A>
__device__ __forceinline__ void stage_fused_ct(float2* tile, A addr, const float2* tw, const Wave& wv) {
    static_assert(Ns * R == L, "the fused stage is the last forward stage");
    const int c = int(threadIdx.x) % C, j = int(threadIdx.x) / C;
    const bool on = j < L / R;
    float2 v[R];
    if (on) {
#pragma unroll
        for (int r = 0; r < R; r++) v[r] = tile[addr(j + r * Ns, c)];
        if constexpr (Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; r++) v[r] = cmul(v[r], tw[r * j]);  // k = j, step = 1
        }
        RegDif<R>::template run<0>(v);
        float2 u[R];
        static_for<0, R>([&](auto rc) {
            constexpr int r = decltype(rc)::value;
            const int kz = j + r * Ns;
            const float psi = wv.a * wv.gz[kz] + wv.b * wv.hz[kz];
            const float2 x = v[dig_rev(R, r)];
            u[r] = make_float2(x.x * psi, -(x.y * psi));
        });
#pragma unroll
        for (int r = 0; r < R; r++) v[r] = u[r];
        RegDif<R>::template run<0>(v);
    }
    __syncthreads();
    if (on) {
        static_for<0, R>([&](auto rc) {
            constexpr int r = decltype(rc)::value;
            tile[addr(j * R + r, c)] = v[dig_rev(R, r)];
        });
    }
    __syncthreads();
}

// A transform policy: the tile FFTs a kernel runs, and its tile width.
// DynFft follows the run-time plan; CtFft<...> is one compile-time plan of at
// most three radices (R2 = 1 for two stages).
struct DynFft {
    static constexpr int kThreads = 512, kMinBlocks = 1;
    static constexpr bool kGlobalTables = false, kBlue = false;
    static constexpr int kMaxLen = CWTHF_MAX_NG / 2;  // longest x pass (the x kernels keep a row in registers)
    static __device__ __forceinline__ int cols(const Plan& p) { return p.C; }
    static __device__ __forceinline__ int len(const Plan& p) { return p.L; }
    static __device__ __forceinline__ int rows(const Plan& p) { return p.L; }
    template <class A>
    static __device__ __forceinline__ void fwd(const Plan& p, float2* t, A addr, const float2* tw) {
        fft_tile(p, t, addr, tw);
    }
    // inverse of conjugated input: conj(DFT(conj(x))) with the conjugations as passes
    template <class A>
    static __device__ __forceinline__ void inv(const Plan& p, float2* t, A addr, const float2* tw) {
        const int n = p.L * p.C;
        for (int i = threadIdx.x; i < n; i += blockDim.x) t[i] = conjf2(t[i]);
        __syncthreads();
        fft_tile(p, t, addr, tw);
        for (int i = threadIdx.x; i < n; i += blockDim.x) t[i] = conjf2(t[i]);
    }
    template <class A>
    static __device__ __forceinline__ void wave(const Plan& p, float2* t, A addr, const float2* tw, const Wave& wv) {
        const int L = p.L, C = p.C, r0 = p.rad[0], r1 = p.rad[1], r2 = p.rad[2];
        if (p.nst == 1) {
            stage_fused(r0, t, addr, tw, L, 1, C, wv);
        } else if (p.nst == 2) {
            stage(r0, t, addr, tw, L, 1, C);
            stage_fused(r1, t, addr, tw, L, r0, C, wv);
            stage(r0, t, addr, tw, L, r1, C);
        } else {
            stage(r0, t, addr, tw, L, 1, C);
            stage(r1, t, addr, tw, L, r0, C);
            stage_fused(r2, t, addr, tw, L, r0 * r1, C, wv);
            stage(r1, t, addr, tw, L, r2, C);
            stage(r0, t, addr, tw, L, r2 * r1, C);
        }
        const int n = L * C;
        for (int i = threadIdx.x; i < n; i += blockDim.x) t[i] = conjf2(t[i]);
    }
};

template <int L_, int C_, int R0, int R1, int R2, int MinBlocks>
struct CtFft {
    static constexpr int kRmin = R2 > 1 ? (R0 < R1 ? (R0 < R2 ? R0 : R2) : (R1 < R2 ? R1 : R2))
                                        : (R1 > 1 ? (R0 < R1 ? R0 : R1) : R0);
    // one butterfly per thread in the smallest-radix stage, and at least one
    // warp per row for the x passes' row loads
    static constexpr int kThreads = C_ * (L_ / kRmin) > 32 * C_ ? C_ * (L_ / kRmin) : 32 * C_;
    static constexpr int kMinBlocks = MinBlocks;
    static constexpr bool kGlobalTables = true;  // y/z pass: tables through the cache
    static constexpr bool kBlue = false;
    static constexpr int kMaxLen = L_;
    static_assert(R0 * R1 * R2 == L_, "radices multiply to the length");
    static __device__ __forceinline__ int cols(const Plan&) { return C_; }
    static __device__ __forceinline__ int len(const Plan&) { return L_; }
    static __device__ __forceinline__ int rows(const Plan&) { return L_; }
    template <bool kCI, bool kCO, class A>
    static __device__ __forceinline__ void run(float2* t, A addr, const float2* tw) {
        if constexpr (R1 == 1) {
            stage_ct<L_, C_, R0, 1, kCI, kCO>(t, addr, tw);
        } else if constexpr (R2 == 1) {
            stage_ct<L_, C_, R0, 1, kCI, false>(t, addr, tw);
            stage_ct<L_, C_, R1, R0, false, kCO>(t, addr, tw);
        } else {
            stage_ct<L_, C_, R0, 1, kCI, false>(t, addr, tw);
            stage_ct<L_, C_, R1, R0, false, false>(t, addr, tw);
            stage_ct<L_, C_, R2, R0 * R1, false, kCO>(t, addr, tw);
        }
    }
    template <class A>
    static __device__ __forceinline__ void fwd(const Plan&, float2* t, A addr, const float2* tw) {
        run<false, false>(t, addr, tw);
    }
    template <class A>
    static __device__ __forceinline__ void inv(const Plan&, float2* t, A addr, const float2* tw) {
        run<true, true>(t, addr, tw);
    }
    template <class A>
    static __device__ __forceinline__ void wave(const Plan&, float2* t, A addr, const float2* tw, const Wave& wv) {
        if constexpr (R1 == 1) {
            static_assert(R1 != 1, "single-stage wavelet plans use the run-time path");
        } else if constexpr (R2 == 1) {
            stage_ct<L_, C_, R0, 1, false, false>(t, addr, tw);
            stage_fused_ct<L_, C_, R1, R0>(t, addr, tw, wv);
            stage_ct<L_, C_, R0, R1, false, true>(t, addr, tw);
        } else {
            stage_ct<L_, C_, R0, 1, false, false>(t, addr, tw);
            stage_ct<L_, C_, R1, R0, false, false>(t, addr, tw);
            stage_fused_ct<L_, C_, R2, R0 * R1>(t, addr, tw, wv);
            stage_ct<L_, C_, R1, R2, false, false>(t, addr, tw);
            stage_ct<L_, C_, R0, R2 * R1, false, true>(t, addr, tw);
        }
    }
};

// Bluestein (chirp-z) policy for a pass length Lb with a prime factor the
// radix stages lack: with nk = (n^2 + k^2 - (k - n)^2) / 2,
//   X_k = conj(b_k) sum_n (x_n conj(b_n)) b_(k-n),   b_n = exp(i pi n^2 / Lb),
// a circular convolution of length L >= 2 Lb - 1 (the run-time plan's length,
// which has radix stages) done as DFT_L, a multiply by the DFT of the wrapped
// chirp, and a conjugated DFT_L.  The tile holds L rows; the pass's Lb rows
// come in and go out through its first rows.  Tables (chirp, transformed
// chirp, twiddles of L) are read through the cache.
struct BlueFft {
    static constexpr int kThreads = 512, kMinBlocks = 1;
    static constexpr bool kGlobalTables = true, kBlue = true;
    static constexpr int kMaxLen = CWTHF_MAX_NG / 2;
    static __device__ __forceinline__ int cols(const Plan& p) { return p.C; }
    static __device__ __forceinline__ int len(const Plan& p) { return p.Lb; }
    static __device__ __forceinline__ int rows(const Plan& p) { return p.L; }
    // DFT_Lb of the tile's first Lb rows (each conjugated on the way in and/or
    // out when asked), in place
    template <bool kConjIn, bool kConjOut, class A>
    static __device__ __forceinline__ void run(const Plan& p, float2* t, A addr, const float2* tw) {
        const int Lb = p.Lb, Mb = p.L, C = p.C;
        // a_n = x_n conj(b_n), zero-padded to Mb rows
        for (int i = threadIdx.x; i < Mb * C; i += blockDim.x) {
            const int l = i / C, c = i - l * C;
            float2 v = make_float2(0.f, 0.f);
            if (l < Lb) {
                v = t[addr(l, c)];
                if (kConjIn) v.y = -v.y;
                v = cmul(v, conjf2(p.chirp[l]));
            }
            t[addr(l, c)] = v;
        }
        __syncthreads();
        fft_tile<true>(p, t, addr, tw);
        // times the transformed chirp (already divided by Mb), conjugated: the
        // second DFT then gives the conjugate of the circular convolution
        for (int i = threadIdx.x; i < Mb * C; i += blockDim.x) {
            const int l = i / C, c = i - l * C;
            t[addr(l, c)] = conjf2(cmul(t[addr(l, c)], p.bhat[l]));
        }
        __syncthreads();
        fft_tile<true>(p, t, addr, tw);
        // X_k = conj(b_k) conv_k = conj(b_k t_k)
        for (int i = threadIdx.x; i < Lb * C; i += blockDim.x) {
            const int l = i / C, c = i - l * C;
            const float2 v = cmul(t[addr(l, c)], p.chirp[l]);
            t[addr(l, c)] = kConjOut ? v : conjf2(v);
        }
        __syncthreads();
    }
    template <class A>
    static __device__ __forceinline__ void fwd(const Plan& p, float2* t, A addr, const float2* tw) {
        run<false, false>(p, t, addr, tw);
    }
    template <class A>
    static __device__ __forceinline__ void inv(const Plan& p, float2* t, A addr, const float2* tw) {
        run<true, true>(p, t, addr, tw);
    }
    // forward, multiply by Psi^ and conjugate, forward, conjugate: the
    // unnormalised inverse of the product
    template <class A>
    static __device__ __forceinline__ void wave(const Plan& p, float2* t, A addr, const float2* tw, const Wave& wv) {
        run<false, false>(p, t, addr, tw);
        const int Lb = p.Lb, C = p.C;
        for (int i = threadIdx.x; i < Lb * C; i += blockDim.x) {  // i % C == threadIdx.x % C: this thread's column
            const int l = i / C, c = i - l * C;
            const float psi = wv.a * wv.gz[l] + wv.b * wv.hz[l];
            const float2 x = t[addr(l, c)];
            t[addr(l, c)] = make_float2(x.x * psi, -(x.y * psi));
        }
        __syncthreads();
        run<false, true>(p, t, addr, tw);
    }
};

// ---------------------------------------------------------------------------
// TMA and mbarrier helpers (inline PTX).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return uint32_t(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// Bounded wait on phase `parity`; returns false if the limit was reached.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit) {
    uint32_t a = smem_u32(bar);
    for (long long it = 0; it < limit; it++) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1, int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, const void* src, int c0, int c1, int c2) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];"
                 ::"l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(src))
                 : "memory");
}
__device__ __forceinline__ void tma_store_commit_and_drain() {
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// ---------------------------------------------------------------------------
// y / z pencil pass: one CTA transforms C adjacent columns of one plane.
// ---------------------------------------------------------------------------
enum YzMode : int { kYzForward = 0, kYzInverse = 1, kYzWavelet = 2 };

struct YzArgs {
    Plan p;
    int ncc;         // column chunks per plane
    int boxr;        // rows per TMA box
    int nbox;        // boxes per tile (boxr * nbox == L; >= L for a Bluestein pass, whose last box may
                     // overhang the end of the axis)
    int mode;
    int along_z;     // 1: transform along z (plane index o = y), 0: along y (o = z)
    int nplanes;     // planes (ng)
    int M;           // ng / 2 (highest valid kx)
    const float2* tw;   // [L]
    const float* ghat;  // [L]  G^(k)   (wavelet mode)
    const float* hhat;  // [L]  H^(k)
    float scale;        // w^1.5 * mass_unit / ng^3
    int* status;
    // fault injection (tests): CTA no_copy_block arms its barrier for the tile
    // but issues no copy, so its bounded wait (no_copy_spin polls) runs out
    // with nothing in flight; -1: off
    int no_copy_block;
    long long no_copy_spin;
};

// One CTA per tile: TMA brings the [L][C] pencil tile into shared memory
// (mbarrier completion), the block transforms it, TMA stores it back.
// Several CTAs per SM overlap their load, compute and store phases.
template <class F>
__global__ void __launch_bounds__(F::kThreads, F::kMinBlocks)
    k_fft_yz(const __grid_constant__ CUtensorMap in_map, const __grid_constant__ CUtensorMap out_map, YzArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const Plan& p = a.p;
    const int L = F::len(p), C = F::cols(p);
    // TMA boxes land at 128-byte aligned offsets of the tile
    unsigned char* base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    float2* tile = reinterpret_cast<float2*>(base);
    // twiddle and wavelet tables: read through the cache (compile-time plans, so
    // that three CTAs fit an SM) or staged in shared memory (run-time plans)
    const float2* tw = a.tw;
    const float* gz = a.ghat;
    const float* hz = a.hhat;
    const int RW = F::rows(p);  // tile rows (more than L for a Bluestein pass)
    uint64_t* bar = reinterpret_cast<uint64_t*>(tile + RW * C);
    if constexpr (!F::kGlobalTables) {
        float2* tws = tile + RW * C;
        float* gzs = reinterpret_cast<float*>(tws + L);
        float* hzs = gzs + L;
        bar = reinterpret_cast<uint64_t*>(hzs + L);  // 8-byte aligned: 8 * (RW*C + 2L) bytes in
        for (int i = threadIdx.x; i < L; i += blockDim.x) {
            tws[i] = a.tw[i];
            if (a.mode == kYzWavelet) {
                gzs[i] = a.ghat[i];
                hzs[i] = a.hhat[i];
            }
        }
        tw = tws;
        gz = gzs;
        hz = hzs;
    }
    const int cc = blockIdx.x % a.ncc, o = blockIdx.x / a.ncc;

    const bool no_copy = int(blockIdx.x) == a.no_copy_block;
    if (threadIdx.x == 0) mbar_init(bar, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        // whole boxes (a Bluestein pass's last box may overhang the axis: the
        // rows past it arrive as zeros and count like the others)
        mbar_expect_tx(bar, uint32_t(a.nbox) * uint32_t(a.boxr) * C * 8u);
        for (int b = 0; b < a.nbox && !no_copy; b++) {
            const int r = b * a.boxr;
            if (a.along_z) tma_load_3d(tile + r * C, &in_map, bar, 2 * cc * C, o, r);
            else tma_load_3d(tile + r * C, &in_map, bar, 2 * cc * C, r, o);
        }
    }
    Wave wv{0.f, 0.f, gz, hz};
    if (a.mode == kYzWavelet) {
        // column c <-> kx = cc*C + c, this plane <-> ky = o
        const int kx = cc * C + int(threadIdx.x % C);
        if (kx <= a.M) {
            const float gx = a.ghat[kx], hx = a.hhat[kx], gy = a.ghat[o], hy = a.hhat[o];
            wv.a = a.scale * (6.f * gx * gy - hx * gy - gx * hy);
            wv.b = -a.scale * gx * gy;
        }
    }
    __syncthreads();
    // the whole block agrees on the outcome of its bounded wait before leaving
    // together.  After a timeout the call's results are unspecified (the status
    // word says so); a copy that is still outstanding gets a second bounded wait.
    const bool loaded = mbar_wait(bar, 0, no_copy ? a.no_copy_spin : kSpinLimit);
    if (__syncthreads_or(!loaded)) {
        if (threadIdx.x == 0) set_status(a.status, CWTHF_E_TIMEOUT);
        if (!no_copy) mbar_wait(bar, 0, kSpinLimit);
        return;
    }
    AddrPlain addr{C};
    if (a.mode == kYzInverse) F::inv(p, tile, addr, tw);
    else if (a.mode == kYzForward) F::fwd(p, tile, addr, tw);
    else F::wave(p, tile, addr, tw, wv);  // forward, multiply, inverse (last stage conjugates)
    fence_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int b = 0; b < a.nbox; b++) {
            const int r = b * a.boxr;
            if (a.along_z) tma_store_3d(&out_map, tile + r * C, 2 * cc * C, o, r);
            else tma_store_3d(&out_map, tile + r * C, 2 * cc * C, r, o);
        }
        tma_store_commit_and_drain();
    }
}

// ---------------------------------------------------------------------------
// x passes: C rows of one real transform each (plain coalesced loads).
// ---------------------------------------------------------------------------
struct XArgs {
    Plan p;          // complex FFT of length M = ng / 2 over C rows
    int ng, M, P;
    int64_t rows;    // ng * ng
    const float2* twM;  // [M]   exp(-2 pi i m / M)  (Bluestein: the inner length's twiddles)
    const float2* twN;  // [ng]  exp(-2 pi i k / ng)
};

template <class F>
__global__ void __launch_bounds__(F::kThreads, F::kMinBlocks) k_fft_x_fwd(XArgs a, const int64_t* __restrict__ grid,
                                                                          float2* __restrict__ spec) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const Plan& p = a.p;
    const int M = F::len(p), C = F::cols(p);
    float2* tile = reinterpret_cast<float2*>(smem_raw);
    float2* tws = tile + F::rows(p) * C;
    double* rowdc = reinterpret_cast<double*>(tws + M);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const float2* tw = tws;
    if constexpr (F::kBlue) tw = a.twM;  // the inner length's twiddles, through the cache
    else
        for (int i = threadIdx.x; i < M; i += blockDim.x) tws[i] = a.twM[i];
    AddrSwz addr{C};
    // load, exact row sum, remove the row's integer mean exactly, round to fp32.
    // Dropping the mean's fractional part only shifts the row's DC bin, which is
    // replaced by the exact row sum below.  The spectrum is in units of 2^-30 of
    // the grid (mass_unit is applied with the wavelet).
    constexpr float kUnit = 9.3132257461547852e-10f;  // 2^-30, exact
    constexpr int kRowVec = (F::kMaxLen + 31) / 32;  // a row's int64 pairs per lane
    for (int r = warp; r < C; r += nwarp) {
        int64_t row = int64_t(blockIdx.x) * C + r;
        longlong2 v[kRowVec];
        long long sum = 0;
        const longlong2* src = reinterpret_cast<const longlong2*>(grid + row * a.ng);
#pragma unroll
        for (int i = 0; i < kRowVec; i++) {
            int k = lane + 32 * i;
            v[i] = (row < a.rows && k < M) ? src[k] : make_longlong2(0, 0);
            sum += v[i].x + v[i].y;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        const long long q0 = sum / a.ng;  // grid values are >= 0
        if (lane == 0) rowdc[r] = double(__ll2float_rn(sum) * kUnit);
#pragma unroll
        for (int i = 0; i < kRowVec; i++) {
            int k = lane + 32 * i;
            if (k < M) {
                float re = __ll2float_rn(v[i].x - q0) * kUnit;
                float im = __ll2float_rn(v[i].y - q0) * kUnit;
                tile[addr(k, r)] = make_float2(re, im);
            }
        }
    }
    __syncthreads();
    F::fwd(p, tile, addr, tw);
    // r2c post-processing: X[k] = (Z[k] + Z*[M-k])/2 - (i/2) W_N^k (Z[k] - Z*[M-k])
    for (int r = warp; r < C; r += nwarp) {
        int64_t row = int64_t(blockIdx.x) * C + r;
        if (row >= a.rows) continue;
        float2* out = spec + row * a.P;
        for (int k = lane; k <= M / 2; k += 32) {
            float2 zk = tile[addr(k, r)];
            float2 zm = tile[addr((M - k) % M, r)];
            if (k == 0) {
                out[0] = make_float2(float(rowdc[r]), 0.f);
                out[M] = make_float2(zk.x - zk.y, 0.f);
                continue;
            }
            float2 w = a.twN[k];
            // k side
            float2 e = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));   // (Z[k] + conj Z[M-k]) / 2
            float2 d = make_float2(0.5f * (zk.x - zm.x), 0.5f * (zk.y + zm.y));   // (Z[k] - conj Z[M-k]) / 2
            float2 wd = cmul(w, d);
            out[k] = make_float2(e.x + wd.y, e.y - wd.x);  // e - i w d
            if (2 * k != M) {
                // M-k side: the same with Z[k] and Z[M-k] swapped and W^(M-k) = -conj(W^k)
                float2 e2 = make_float2(e.x, -e.y);
                float2 d2 = make_float2(-d.x, d.y);
                float2 w2 = make_float2(-w.x, w.y);
                float2 wd2 = cmul(w2, d2);
                out[M - k] = make_float2(e2.x + wd2.y, e2.y - wd2.x);
            }
        }
        for (int k = M + 1 + lane; k < a.P; k += 32) out[k] = make_float2(0.f, 0.f);
    }
}

template <class F>
__global__ void __launch_bounds__(F::kThreads, F::kMinBlocks) k_fft_x_inv(XArgs a, const float2* __restrict__ spec,
                                                                          float* __restrict__ cwt) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const Plan& p = a.p;
    const int M = F::len(p), C = F::cols(p);
    float2* tile = reinterpret_cast<float2*>(smem_raw);
    float2* tws = tile + F::rows(p) * C;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const float2* tw = tws;
    if constexpr (F::kBlue) tw = a.twM;
    else
        for (int i = threadIdx.x; i < M; i += blockDim.x) tws[i] = a.twM[i];
    AddrSwz addr{C};
    // c2r pre-processing: Z'[k] = (X[k] + X*[M-k]) + i W_N^-k (X[k] - X*[M-k]); stored conjugated.
    // All of a row's loads are issued before any is used (memory parallelism).
    for (int r = warp; r < C; r += nwarp) {
        int64_t row = int64_t(blockIdx.x) * C + r;
        const float2* in = spec + (row < a.rows ? row : 0) * a.P;
        constexpr int kPairs = F::kMaxLen / 64 + 1;  // k = lane + 32 i covers k <= M/2
        float2 xk[kPairs], xm[kPairs];
#pragma unroll
        for (int i = 0; i < kPairs; i++) {
            const int k = lane + 32 * i;
            if (k <= M / 2) {
                xk[i] = in[k];
                xm[i] = in[M - k];
            }
        }
#pragma unroll
        for (int i = 0; i < kPairs; i++) {
            const int k = lane + 32 * i;
            if (k > M / 2) continue;
            float2 a0 = xk[i], a1 = xm[i];
            if (k == 0) {
                a0.y = 0.f;
                a1.y = 0.f;
            }
            float2 e = make_float2(a0.x + a1.x, a0.y - a1.y);  // X[k] + conj X[M-k]
            float2 d = make_float2(a0.x - a1.x, a0.y + a1.y);  // X[k] - conj X[M-k]
            float2 winv = conjf2(a.twN[k]);                     // W_N^-k
            float2 wd = cmul(winv, d);
            float2 zk = make_float2(e.x - wd.y, e.y + wd.x);   // e + i W^-k d
            tile[addr(k, r)] = conjf2(zk);
            if (k != 0 && 2 * k != M) {
                float2 e2 = make_float2(e.x, -e.y);
                float2 d2 = make_float2(-d.x, d.y);
                float2 w2 = make_float2(-winv.x, winv.y);      // W_N^-(M-k) = -conj(W_N^-k)
                float2 wd2 = cmul(w2, d2);
                float2 zm = make_float2(e2.x - wd2.y, e2.y + wd2.x);
                tile[addr(M - k, r)] = conjf2(zm);
            }
        }
    }
    __syncthreads();
    F::fwd(p, tile, addr, tw);
    for (int r = warp; r < C; r += nwarp) {
        int64_t row = int64_t(blockIdx.x) * C + r;
        if (row >= a.rows) continue;
        float2* out = reinterpret_cast<float2*>(cwt + row * a.ng);
        for (int n = lane; n < M; n += 32) {
            float2 z = tile[addr(n, r)];
            out[n] = make_float2(z.x, -z.y);  // conj back; z[n] = x[2n] + i x[2n+1]
        }
    }
}

// ---------------------------------------------------------------------------
// Host side: plans, tables, tensor maps, launches.
// ---------------------------------------------------------------------------
constexpr int kRadices[] = {2, 3, 4, 5, 6, 7, 8, 9, 10, 12, 14, 15, 16, 18, 20, 21, 24, 25, 27, 28, 30, 32};

bool is_radix(int r) {
    for (int x : kRadices)
        if (x == r) return true;
    return false;
}

// Up to three radices from kRadices whose product is L, maximising the
// smallest radix (fewest threads, least shared-memory traffic).
bool make_plan(int L, Plan& p) {
    int best = -1;
    p.L = L;
    if (is_radix(L)) {
        p.nst = 1;
        p.rad[0] = L;
        return true;
    }
    for (int a : kRadices) {
        if (L % a) continue;
        int rem = L / a;
        if (is_radix(rem) && std::min(a, rem) > best) {
            best = std::min(a, rem);
            p.nst = 2;
            p.rad[0] = a;
            p.rad[1] = rem;
        }
    }
    if (best > 0) return true;
    for (int a : kRadices)
        for (int b : kRadices) {
            if (L % (a * b)) continue;
            int c = L / (a * b);
            if (!is_radix(c)) continue;
            int m = std::min(a, std::min(b, c));
            if (m > best) {
                best = m;
                p.nst = 3;
                p.rad[0] = a;
                p.rad[1] = b;
                p.rad[2] = c;
            }
        }
    return best > 0;
}

// A pass of length L runs its radix plan if one fits the kernel (fit picks
// the tile width); otherwise it runs as a Bluestein pass whose inner length is
// the smallest Mb >= 2 L - 1 (and at most 2.25 L + 64) with a radix plan that fits.
template <class Fit>
bool pass_plan_for(int L, Plan& p, Fit&& fit) {
    p.Lb = 0;
    if (make_plan(L, p) && fit(p)) return true;
    for (int Mb = 2 * L - 1; Mb <= 2 * L + L / 4 + 64; Mb++) {
        p.Lb = 0;
        if (!make_plan(Mb, p)) continue;
        p.Lb = L;
        if (fit(p)) return true;
    }
    p.Lb = 0;
    return false;
}

int plan_threads(const Plan& p) {
    int rmin = 64;
    for (int s = 0; s < p.nst; s++) rmin = std::min(rmin, p.rad[s]);
    int t = p.C * (p.L / rmin);
    return (t + 31) / 32 * 32;
}

// Rows per TMA box for a y/z tile of C columns: the largest divisor of L (at
// most 256) whose box spans a multiple of 128 bytes; else, for a tile of
// `rows` >= L rows (a Bluestein pass), the largest such box whose whole boxes
// fit the tile, the last one overhanging the end of the axis (its loads read
// zeros there and its stores are clipped); else -1.
int pick_boxr(int L, int C, int rows = 0) {
    for (int b = std::min(L, 256); b >= 1; b--)
        if (L % b == 0 && (size_t(b) * C * 8) % 128 == 0) return b;
    for (int b = std::min(L, 256); b >= 1 && rows >= L; b--)
        if ((size_t(b) * C * 8) % 128 == 0 && div_up(L, b) * b <= rows) return b;
    return -1;
}
int plan_boxr(int L, const Plan& p) { return pick_boxr(L, p.C, p.Lb ? p.L : 0); }

// A Bluestein tile of q.C columns may run its stages with two butterflies per
// thread (BlueFft, 512 threads): every stage fits in 2 T butterflies, and a
// stage that needs two per thread has a radix of at most 16.
bool two_per_thread_ok(const Plan& q, int T) {
    for (int st = 0; st < q.nst; st++) {
        const int nb = q.C * (q.L / q.rad[st]);
        if (nb > 2 * T || (nb > T && q.rad[st] > 16)) return false;
    }
    return true;
}

// Tile width of a Bluestein pass: four or more columns with one butterfly per
// thread (<= 256, then <= 512 threads, <= 64 KB), else four or more with two
// butterflies per thread (512 threads, <= 96 KB: three CTAs per SM), else two
// columns.  Wider tiles move longer row segments per TMA box (two columns are
// 16 bytes per row).  min_threads(C) is the pass's own least block size,
// `fits` its other constraints.
template <class MinT, class Fits>
bool bluestein_tile(Plan& q, MinT&& min_threads, Fits&& fits) {
    for (int tmax : {256, 512})
        for (int C : {16, 8, 4}) {
            q.C = C;
            q.T = std::max(plan_threads(q), min_threads(C));
            if (size_t(q.L) * C * 8 <= 65536 && q.T <= tmax && fits(q)) return true;
        }
    for (int C : {16, 8, 4}) {
        q.C = C;
        q.T = std::max(std::min(plan_threads(q), 512), min_threads(C));
        if (size_t(q.L) * C * 8 <= 98304 && q.T <= 512 && two_per_thread_ok(q, q.T) && fits(q)) return true;
    }
    q.C = 2;
    q.T = std::max(plan_threads(q), min_threads(2));
    return size_t(q.L) * 2 * 8 <= 65536 && q.T <= 512 && fits(q);
}

// Columns per y/z tile: <= 64 KB of complex data and a valid TMA box,
// preferring <= 256 threads (two CTAs per SM at 128 registers) over <= 512
// (Bluestein passes: bluestein_tile).
bool yz_plan(int L, Plan& p) {
    return pass_plan_for(L, p, [L](Plan& q) {
        if (q.Lb)
            return bluestein_tile(q, [](int) { return 0; }, [L](const Plan& r) { return plan_boxr(L, r) > 0; });
        for (int tmax : {256, 512})
            for (int C : {16, 8, 4, 2}) {
                q.C = C;
                q.T = plan_threads(q);
                if (size_t(q.L) * C * 8 <= 65536 && q.T <= tmax && plan_boxr(L, q) > 0) return true;
            }
        return false;
    });
}

// Rows per x tile: <= 64 KB of complex data, one warp per row for the loads,
// preferring <= 256 threads (two CTAs per SM) over <= 512.
bool x_plan(int M, Plan& p) {
    return pass_plan_for(M, p, [](Plan& q) {
        if (q.Lb)  // at least one warp per row for the row loads
            return bluestein_tile(q, [](int C) { return 32 * std::min(C, 16); }, [](const Plan&) { return true; });
        for (int tmax : {256, 512})
            for (int C : {16, 8, 4, 2}) {
                q.C = C;
                q.T = std::max(plan_threads(q), 32 * std::min(C, 16));
                if (size_t(q.L) * C * 8 <= 65536 && q.T <= tmax) return true;
            }
        return false;
    });
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    });
    return fn;
}

// 3D view of a spectrum as floats: dim0 = 2P floats (contiguous), dim1 = y,
// dim2 = z.  A box is C complex columns by boxr rows of the transform axis
// (y: {2C, boxr, 1}; z: {2C, 1, boxr}); either lands in shared memory as a
// dense [boxr][C] complex tile.
int make_spec_map(CUtensorMap* map, float2* base, int ng, bool along_z, int C, int boxr) {
    auto fn = encode_fn();
    if (!fn) return CWTHF_E_CUDA;
    const int P = spec_pitch(ng);
    cuuint64_t dims[3] = {cuuint64_t(2 * P), cuuint64_t(ng), cuuint64_t(ng)};
    cuuint64_t row = cuuint64_t(P) * 8, plane = row * ng;
    cuuint64_t strides[2] = {row, plane};
    cuuint32_t box[3] = {cuuint32_t(2 * C), along_z ? 1u : cuuint32_t(boxr), along_z ? cuuint32_t(boxr) : 1u};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? CWTHF_OK : CWTHF_E_CUDA;
}

size_t yz_smem(const Plan& p, bool global_tables) {
    return 128 + size_t(p.L) * p.C * 8 + (global_tables ? 0 : size_t(p.L) * 16) + 16;
}
size_t x_smem(const Plan& p) { return size_t(p.L) * p.C * 8 + size_t(p.L) * 8 + size_t(p.C) * 8; }

void host_twiddles(int n, std::vector<float2>& out) {
    out.resize(n);
    for (int m = 0; m < n; m++) {
        double ang = 2.0 * kPi * double(m) / double(n);
        out[m] = make_float2(float(std::cos(ang)), float(-std::sin(ang)));
    }
}

// The twiddle table of a grid size: twN [ng] and twM [ng/2], then for each
// Bluestein pass its chirp, transformed chirp and inner twiddles (float
// offsets; 0 = absent).
struct TwLayout {
    size_t n = 0;
    size_t chirp_yz = 0, bhat_yz = 0, tw_yz = 0, chirp_x = 0, bhat_x = 0, tw_x = 0;
    int lb_yz = 0, mb_yz = 0, lb_x = 0, mb_x = 0;
};
TwLayout tw_layout(int ng) {
    TwLayout t;
    size_t o = 3 * size_t(ng);
    Plan p;
    if (yz_plan(ng, p) && p.Lb) {
        t.lb_yz = p.Lb;
        t.mb_yz = p.L;
        t.chirp_yz = o;
        o += 2 * size_t(p.Lb);
        t.bhat_yz = o;
        o += 2 * size_t(p.L);
        t.tw_yz = o;
        o += 2 * size_t(p.L);
    }
    if (x_plan(ng / 2, p) && p.Lb) {
        t.lb_x = p.Lb;
        t.mb_x = p.L;
        t.chirp_x = o;
        o += 2 * size_t(p.Lb);
        t.bhat_x = o;
        o += 2 * size_t(p.L);
        t.tw_x = o;
        o += 2 * size_t(p.L);
    }
    t.n = o;
    return t;
}

// Bluestein tables in fp64, stored as fp32: the chirp b_n = exp(i pi n^2 / Lb),
// n < Lb (n^2 reduced mod 2 Lb exactly); the DFT of length Mb of the wrapped
// chirp (b_n at n and at Mb - n, zero between), divided by Mb; the twiddles of Mb.
void host_bluestein(int Lb, int Mb, float* chirp, float* bhat, float* tw) {
    std::vector<double> br(Lb), bi(Lb);
    for (int n = 0; n < Lb; n++) {
        const long long q = (static_cast<long long>(n) * n) % (2LL * Lb);
        const double ang = kPi * double(q) / double(Lb);
        br[n] = std::cos(ang);
        bi[n] = std::sin(ang);
        chirp[2 * n] = float(br[n]);
        chirp[2 * n + 1] = float(bi[n]);
    }
    std::vector<double> cm(Mb), sm(Mb);
    for (int m = 0; m < Mb; m++) {
        cm[m] = std::cos(2.0 * kPi * double(m) / double(Mb));
        sm[m] = std::sin(2.0 * kPi * double(m) / double(Mb));
    }
    for (int k = 0; k < Mb; k++) {
        double sr = 0.0, si = 0.0;
        auto add = [&](int n, int j) {  // B_n = b_j, times exp(-2 pi i n k / Mb)
            const int e = int((static_cast<long long>(n) * k) % Mb);
            sr += br[j] * cm[e] + bi[j] * sm[e];
            si += bi[j] * cm[e] - br[j] * sm[e];
        };
        for (int n = 0; n < Lb; n++) add(n, n);
        for (int n = Mb - Lb + 1; n < Mb; n++) add(n, Mb - n);
        bhat[2 * k] = float(sr / Mb);
        bhat[2 * k + 1] = float(si / Mb);
    }
    std::vector<float2> w;
    host_twiddles(Mb, w);
    std::memcpy(tw, w.data(), w.size() * 8);
}

// G^(k) and H^(k), k < ng: 1D DFTs (real, even sequences) of the sampled
// Gaussian factor and of its w^2 u^2 multiple, in fp64, stored as fp32
// (out[k] = G^(k), out[ng + k] = H^(k)).
void host_wavelet_tables(int ng, double L, double w, float* out) {
    const double dx = L / ng;
    std::vector<double> gn(ng), hn(ng), cosn(ng);
    for (int n = 0; n < ng; n++) {
        int d = (2 * n <= ng) ? n : n - ng;
        double u2 = (dx * d) * (dx * d);
        gn[n] = std::exp(-0.25 * w * w * u2);
        hn[n] = w * w * u2 * gn[n];
        cosn[n] = std::cos(2.0 * kPi * double(n) / double(ng));
    }
    for (int k = 0; k < ng; k++) {
        double sg = 0.0, sh = 0.0;
        for (int n = 0; n < ng; n++) {
            double c = cosn[(int64_t(k) * n) % ng];
            sg += gn[n] * c;
            sh += hn[n] * c;
        }
        out[k] = float(sg);
        out[ng + k] = float(sh);
    }
}

// The context's table slots (allocated by cwthf_create, never grown).  A
// miss fills a slot on the host (the slot's pinned staging) and queues one
// copy to the device on the call's stream, so a call allocates nothing and
// never waits for the device, except when it must reuse a slot whose
// previous copy may still be pending.  Slots read by work captured into a
// CUDA graph are never reused.  A captured call records the copy of a table
// that no uncaptured call has put on the device yet, so such a graph brings
// its own tables on every replay; a table already copied by an uncaptured
// call (cwthf_prepare, or an earlier call) is only read, and that copy must
// be complete before the graph runs.  An uncaptured call that finds a slot
// filled only inside a capture queues the copy itself.  During a capture only
// free slots can be filled; with none left the call fails with
// CWTHF_E_TABLE_CACHE.
int table_lookup(cwthf_ctx* ctx, int kind, int ng, double L, double w, cudaStream_t s, const float** out) {
    std::lock_guard<std::mutex> g(ctx->table_mu);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return CWTHF_E_CUDA;
    const bool capturing = cap != cudaStreamCaptureStatusNone;
    const size_t stride = ctx->table_slot_floats;
    const TwLayout lay = kind == kTableTwiddles ? tw_layout(ng) : TwLayout();
    const size_t n = kind == kTableTwiddles ? lay.n : 2 * size_t(ng);
    if (n > stride) return CWTHF_E_UNSUPPORTED_SIZE;
    int pick = -1;
    for (int i = 0; i < kTableSlots && pick < 0; i++) {
        const TableSlot& t = ctx->table_slot[i];
        if (t.kind == kind && t.ng == ng && t.L == L && t.w == w) pick = i;
    }
    bool fill = pick < 0;
    if (fill) {
        for (int i = 0; i < kTableSlots && pick < 0; i++)
            if (ctx->table_slot[i].kind < 0) pick = i;
        if (pick < 0 && !capturing)  // least recently used slot that no graph reads
            for (int i = 0; i < kTableSlots; i++) {
                const TableSlot& t = ctx->table_slot[i];
                if (!t.graph_ref && (pick < 0 || t.last_use < ctx->table_slot[pick].last_use)) pick = i;
            }
        if (pick < 0) return CWTHF_E_TABLE_CACHE;
    }
    TableSlot& t = ctx->table_slot[pick];
    float* host = ctx->table_host + pick * stride;
    float* dev = ctx->table_dev + pick * stride;
    if (fill) {
        // an evicted slot (only ever filled outside a capture): its last copy
        // must have read the staging before the staging is rewritten
        if (t.kind >= 0 && cudaEventSynchronize(t.filled) != cudaSuccess) return CWTHF_E_CUDA;
        t = TableSlot{-1, 0, 0.0, 0.0, 0, false, false, t.filled};
        if (kind == kTableTwiddles) {  // exp(-2 pi i m / ng), m < ng, then exp(-2 pi i m / (ng/2)), m < ng/2
            std::vector<float2> a, b;
            host_twiddles(ng, a);
            host_twiddles(ng / 2, b);
            std::memcpy(host, a.data(), a.size() * 8);
            std::memcpy(host + 2 * ng, b.data(), b.size() * 8);
            if (lay.lb_yz)
                host_bluestein(lay.lb_yz, lay.mb_yz, host + lay.chirp_yz, host + lay.bhat_yz, host + lay.tw_yz);
            if (lay.lb_x) host_bluestein(lay.lb_x, lay.mb_x, host + lay.chirp_x, host + lay.bhat_x, host + lay.tw_x);
        } else {
            host_wavelet_tables(ng, L, w, host);
        }
        t.kind = kind;
        t.ng = ng;
        t.L = L;
        t.w = w;
        ctx->table_fills++;
    }
    // a captured call that finds the table already on the device (an earlier
    // uncaptured copy) records no copy: the graph reads the slot, which is
    // kept from now on; otherwise the graph carries the copy itself
    if (!t.on_device) {  // a fill always clears on_device
        if (cudaMemcpyAsync(dev, host, n * 4, cudaMemcpyHostToDevice, s) != cudaSuccess) return CWTHF_E_CUDA;
        if (!capturing) {
            if (cudaEventRecord(t.filled, s) != cudaSuccess) return CWTHF_E_CUDA;
            t.on_device = true;
        }
    }
    t.graph_ref |= capturing;
    t.last_use = ++ctx->table_clock;
    *out = dev;
    return CWTHF_OK;
}

int get_tables(cwthf_ctx* ctx, int ng, cudaStream_t s, Tables& t) {
    const float* p = nullptr;
    int rc = table_lookup(ctx, kTableTwiddles, ng, 0.0, 0.0, s, &p);
    if (rc) return rc;
    t.ng = ng;
    t.twN = reinterpret_cast<const float2*>(p);
    t.twM = reinterpret_cast<const float2*>(p + 2 * ng);
    const TwLayout lay = tw_layout(ng);
    auto at = [&](size_t o) { return o ? reinterpret_cast<const float2*>(p + o) : nullptr; };
    t.chirp_yz = at(lay.chirp_yz);
    t.bhat_yz = at(lay.bhat_yz);
    t.tw_yz = at(lay.tw_yz);
    t.chirp_x = at(lay.chirp_x);
    t.bhat_x = at(lay.bhat_x);
    t.tw_x = at(lay.tw_x);
    return CWTHF_OK;
}

// Compile-time instances for the plans of the large power-of-two grids; any
// other plan runs the run-time kernels.  An instance is used only when the
// run-time plan picks exactly its length, tile width and radices.
template <class F>
bool plan_is(const Plan& p, int L, int C, int r0, int r1, int r2) {
    const int nst = r2 > 1 ? 3 : (r1 > 1 ? 2 : 1);
    return p.L == L && p.C == C && p.nst == nst && p.rad[0] == r0 && (nst < 2 || p.rad[1] == r1) &&
           (nst < 3 || p.rad[2] == r2) && p.T == F::kThreads;
}
using Yz1024 = CtFft<1024, 8, 32, 32, 1, 3>;
using Yz512 = CtFft<512, 8, 16, 32, 1, 3>;
using X512 = CtFft<512, 8, 16, 32, 1, 3>;
using X256 = CtFft<256, 8, 16, 16, 1, 3>;

using YzKernel = void (*)(const CUtensorMap, const CUtensorMap, YzArgs);
YzKernel pick_yz(const Plan& p, bool& global_tables) {
    global_tables = true;
    if (p.Lb) return k_fft_yz<BlueFft>;
    if (plan_is<Yz1024>(p, 1024, 8, 32, 32, 1)) return k_fft_yz<Yz1024>;
    if (plan_is<Yz512>(p, 512, 8, 16, 32, 1)) return k_fft_yz<Yz512>;
    global_tables = false;
    return k_fft_yz<DynFft>;
}
using XFwdKernel = void (*)(XArgs, const int64_t*, float2*);
using XInvKernel = void (*)(XArgs, const float2*, float*);
XFwdKernel pick_x_fwd(const Plan& p) {
    if (p.Lb) return k_fft_x_fwd<BlueFft>;
    if (plan_is<X512>(p, 512, 8, 16, 32, 1)) return k_fft_x_fwd<X512>;
    if (plan_is<X256>(p, 256, 8, 16, 16, 1)) return k_fft_x_fwd<X256>;
    return k_fft_x_fwd<DynFft>;
}
XInvKernel pick_x_inv(const Plan& p) {
    if (p.Lb) return k_fft_x_inv<BlueFft>;
    if (plan_is<X512>(p, 512, 8, 16, 32, 1)) return k_fft_x_inv<X512>;
    if (plan_is<X256>(p, 256, 8, 16, 16, 1)) return k_fft_x_inv<X256>;
    return k_fft_x_inv<DynFft>;
}

// A caller's plan (which = 0: y/z passes of length ng, 1: x passes of length
// ng/2), checked against what the kernels can run: radices from kRadices
// whose product is the length, C in {2, 4, 8, 16}, <= 64 KB of tile, <= 512
// threads, and for the y/z passes a valid TMA box.
bool plan_from(int L, int which, int C, const int* rad, int nst, Plan& p) {
    if (nst < 1 || nst > 3 || !(C == 2 || C == 4 || C == 8 || C == 16)) return false;
    int prod = 1;
    for (int i = 0; i < nst; i++) {
        if (!is_radix(rad[i])) return false;
        prod *= rad[i];
    }
    if (prod != L) return false;
    p.L = L;
    p.nst = nst;
    for (int i = 0; i < 3; i++) p.rad[i] = i < nst ? rad[i] : 1;
    p.C = C;
    p.T = which == 0 ? plan_threads(p) : std::max(plan_threads(p), 32 * std::min(C, 16));
    if (size_t(L) * C * 8 > 65536 || p.T > 512) return false;
    return which != 0 || pick_boxr(L, C) > 0;
}

// The plan a pass of this context uses: the caller's, else the built-in rule.
bool pass_plan(cwthf_ctx* ctx, int ng, int which, Plan& p) {
    {
        std::lock_guard<std::mutex> g(ctx->table_mu);
        for (const auto& o : ctx->fft_plans)
            if (o.ng == ng && o.which == which) return plan_from(which == 0 ? ng : ng / 2, which, o.C, o.rad, o.nst, p);
    }
    return which == 0 ? yz_plan(ng, p) : x_plan(ng / 2, p);
}

int launch_yz(cwthf_ctx* ctx, float2* src, float2* dst, int ng, bool along_z, int mode, const Tables* t,
              const float* wtab, double w, double mass_unit, cudaStream_t s) {
    Plan p;
    if (!pass_plan(ctx, ng, 0, p)) return CWTHF_E_UNSUPPORTED_SIZE;
    int boxr = plan_boxr(ng, p);
    if (boxr < 0) return CWTHF_E_UNSUPPORTED_SIZE;
    if (p.Lb && !(t->chirp_yz && t->bhat_yz && t->tw_yz)) return CWTHF_E_UNSUPPORTED_SIZE;
    p.chirp = t->chirp_yz;
    p.bhat = t->bhat_yz;
    CUtensorMap in_map, out_map;
    int rc = make_spec_map(&in_map, src, ng, along_z, p.C, boxr);
    if (!rc) rc = make_spec_map(&out_map, dst, ng, along_z, p.C, boxr);
    if (rc) return rc;
    YzArgs a;
    a.p = p;
    a.M = ng / 2;
    a.ncc = div_up(a.M + 1, p.C);
    a.boxr = boxr;
    a.nbox = div_up(ng, boxr);
    a.mode = mode;
    a.along_z = along_z ? 1 : 0;
    a.nplanes = ng;
    a.tw = p.Lb ? t->tw_yz : t->twN;
    a.ghat = wtab;
    a.hhat = wtab ? wtab + ng : nullptr;
    // w^1.5 (Eq. 4), the 1/ng^3 of the inverse DFT, and the mass of one spectrum
    // unit (the x pass already scaled the int64 grid by 2^-30: units of mass_unit)
    a.scale = float(std::pow(w, 1.5) * mass_unit / (double(ng) * ng * ng));
    a.status = ctx->d_status;
    a.no_copy_block = -1;
    a.no_copy_spin = 0;
    if (ctx->dbg_tma_no_copy) {  // one-shot fault injection (cwthf_debug_set)
        ctx->dbg_tma_no_copy = 0;
        a.no_copy_block = 0;
        a.no_copy_spin = 1 << 12;
    }
    bool global_tables = false;
    YzKernel k = pick_yz(p, global_tables);
    size_t smem = yz_smem(p, global_tables);
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    CWTHF_LAUNCH(ctx, s, "k_fft_yz", k<<<unsigned(a.ncc) * ng, p.T, smem, s>>>(in_map, out_map, a));
    return cuda_status(cudaGetLastError());
}

int x_args(cwthf_ctx* ctx, int ng, const Tables* t, XArgs& a) {
    Plan p;
    if (!pass_plan(ctx, ng, 1, p)) return CWTHF_E_UNSUPPORTED_SIZE;
    if (p.Lb && !(t->chirp_x && t->bhat_x && t->tw_x)) return CWTHF_E_UNSUPPORTED_SIZE;
    p.chirp = t->chirp_x;
    p.bhat = t->bhat_x;
    a.p = p;
    a.ng = ng;
    a.M = ng / 2;
    a.P = spec_pitch(ng);
    a.rows = int64_t(ng) * ng;
    a.twM = p.Lb ? t->tw_x : t->twM;
    a.twN = t->twN;
    return CWTHF_OK;
}

}  // namespace

int transform_forward_xy(cwthf_ctx* ctx, const int64_t* grid, int ng, float2* spec, cudaStream_t s) {
    if (ng > CWTHF_MAX_NG) return CWTHF_E_UNSUPPORTED_SIZE;
    Tables tb;
    int rc = get_tables(ctx, ng, s, tb);
    if (rc) return rc;
    const Tables* t = &tb;
    XArgs a;
    rc = x_args(ctx, ng, t, a);
    if (rc) return rc;
    XFwdKernel k = pick_x_fwd(a.p);
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(x_smem(a.p)));
    CWTHF_LAUNCH(ctx, s, "k_fft_x_fwd", k<<<div_up(a.rows, a.p.C), a.p.T, x_smem(a.p), s>>>(a, grid, spec));
    if ((rc = cuda_status(cudaGetLastError()))) return rc;
    return launch_yz(ctx, spec, spec, ng, false, kYzForward, t, nullptr, 0.0, 1.0, s);
}

int transform_tables(cwthf_ctx* ctx, int ng, double L, const double* w, int n, const float** wtab,
                     cudaStream_t s) {
    if (n + 1 > kTableSlots) return CWTHF_E_TABLE_CACHE;
    Tables tb;
    int rc = get_tables(ctx, ng, s, tb);
    for (int i = 0; i < n && !rc; i++) rc = table_lookup(ctx, kTableWavelet, ng, L, w[i], s, &wtab[i]);
    return rc;
}

int transform_wavelet_inverse(cwthf_ctx* ctx, float2* src, float2* dst, int ng, double L, double w,
                              double mass_unit, const float* wtab, float* cwt, cudaStream_t s) {
    Tables tb;
    int rc = get_tables(ctx, ng, s, tb);
    if (rc) return rc;
    const Tables* t = &tb;
    rc = launch_yz(ctx, src, dst, ng, true, kYzWavelet, t, wtab, w, mass_unit, s);
    if (!rc) rc = launch_yz(ctx, dst, dst, ng, false, kYzInverse, t, nullptr, 0.0, 1.0, s);
    if (rc) return rc;
    XArgs a;
    if ((rc = x_args(ctx, ng, t, a))) return rc;
    XInvKernel k = pick_x_inv(a.p);
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(x_smem(a.p)));
    CWTHF_LAUNCH(ctx, s, "k_fft_x_inv", k<<<div_up(a.rows, a.p.C), a.p.T, x_smem(a.p), s>>>(a, dst, cwt));
    return cuda_status(cudaGetLastError());
}

int set_fft_plan(cwthf_ctx* ctx, int ng, int which, int C, const int* rad, int nst) {
    if (which != 0 && which != 1) return CWTHF_E_INVALID_ARG;
    std::lock_guard<std::mutex> g(ctx->table_mu);
    auto& v = ctx->fft_plans;
    v.erase(std::remove_if(v.begin(), v.end(), [&](const cwthf_ctx::PlanOverride& o) {
                return o.ng == ng && o.which == which;
            }), v.end());
    if (nst == 0) return CWTHF_OK;  // back to the built-in rule
    Plan p;
    if (!rad || !plan_from(which == 0 ? ng : ng / 2, which, C, rad, nst, p)) return CWTHF_E_INVALID_ARG;
    cwthf_ctx::PlanOverride o{ng, which, C, nst, {1, 1, 1}};
    for (int i = 0; i < nst; i++) o.rad[i] = rad[i];
    v.push_back(o);
    return CWTHF_OK;
}

// The same plans and TMA box the launches use: the y/z pass's tile width
// decides the box, the x passes have a plan of their own.
bool fft_size_supported(int ng) {
    Plan yz, x;
    return (ng % 2 == 0) && ng <= CWTHF_MAX_NG && yz_plan(ng, yz) && plan_boxr(ng, yz) > 0 && x_plan(ng / 2, x);
}

void free_tables(cwthf_ctx* ctx) {
    for (TableSlot& t : ctx->table_slot) {
        if (t.filled) cudaEventDestroy(t.filled);
        t = TableSlot();
    }
}

int init_tables(cwthf_ctx* ctx) {
    for (TableSlot& t : ctx->table_slot)
        if (cudaEventCreateWithFlags(&t.filled, cudaEventDisableTiming) != cudaSuccess) return CWTHF_E_CUDA;
    return CWTHF_OK;
}

}  // namespace cwthf
