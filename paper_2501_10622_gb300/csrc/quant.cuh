// quant.cuh -- the fixed-point position and mass rules shared by the deposit
// and the particle assignment (one definition, so both stages agree bit for bit).
#pragma once
#include <cmath>

#include "internal.cuh"

namespace cwthf {

struct DepArgs {
    const float* pos;
    const float* mass;
    double mass_unit;
    uint32_t scale_m;  // quantisation scale s = scale_m * 2^scale_e (scale_m < 2^29)
    int scale_e;
    int64_t modulus;   // ng * 2^10
    int64_t np;
    int ng, ntx, nty, ntz;
};

// The quantisation scale N * 2^10 / L: the fp64 quotient N/L times 2^10,
// rounded to 29 significant bits (half to even), as an integer mantissa and
// a power of two.  With 24-bit float positions the product x * s then has at
// most 53 significant bits: it is exact, in fp64 and in 64-bit integers.
inline void quant_scale(int ng, double L, uint32_t& m, int& e) {
    double s = (double(ng) / L) * double(kFracOne);
    int ex;
    double f = std::frexp(s, &ex);  // s = f 2^ex, 0.5 <= f < 1
    double mm = std::nearbyint(std::ldexp(f, 29));
    m = uint32_t(mm);
    e = ex - 29;
    if (m == (1u << 29)) {  // rounded up to the next power of two
        m >>= 1;
        e += 1;
    }
}

inline DepArgs make_dep_args(const float* pos, const float* mass, double mass_unit, int64_t np, double L, int ng) {
    DepositGeom g = deposit_geom(ng);
    DepArgs a;
    a.pos = pos;
    a.mass = mass;
    a.mass_unit = mass_unit;
    quant_scale(ng, L, a.scale_m, a.scale_e);
    a.modulus = int64_t(ng) * kFracOne;
    a.np = np;
    a.ng = ng;
    a.ntx = g.ntx;
    a.nty = g.nty;
    a.ntz = g.ntz;
    return a;
}

// floor(x * s) mod ng*2^10 for s = sm * 2^se, evaluated exactly with one
// 32x32 -> 64-bit integer product of the mantissas (no floating point);
// false for non-finite x or |x * s| >= 2^40.
__device__ __forceinline__ bool quantise(float x, uint32_t sm, int se, int64_t modulus, int64_t& q) {
    const uint32_t b = __float_as_uint(x);
    const uint32_t eb = (b >> 23) & 0xffu;
    if (eb == 0xffu) return false;  // infinity or NaN
    uint32_t man = b & 0x7fffffu;
    int ex = -149;  // zero and subnormals: |x| = man * 2^-149
    if (eb) {
        man |= 0x800000u;
        ex = int(eb) - 150;
    }
    const unsigned long long P = (unsigned long long)man * sm;  // |x * s| = P * 2^k, P < 2^53
    const int k = ex + se;
    unsigned long long fl;  // floor(|x * s|)
    bool frac = false;
    if (P == 0) {
        fl = 0;
    } else if (k >= 0) {
        if (k >= 40 || (P >> (40 - k)) != 0) return false;
        fl = P << k;
    } else if (-k >= 64) {
        fl = 0;
        frac = true;
    } else {
        fl = P >> (-k);
        frac = (P & ((1ull << (-k)) - 1ull)) != 0;
    }
    if (fl >= (1ull << 40)) return false;
    int64_t v = (b >> 31) ? -int64_t(fl) - (frac ? 1 : 0) : int64_t(fl);
    if (v < 0 || v >= modulus) {  // outside the box: wrap (rare)
        v %= modulus;
        if (v < 0) v += modulus;
    }
    q = v;
    return true;
}

// Integer mass of particle i: 1 when masses are equal, else rint(m / mass_unit)
// (round half to even).  Returns CWTHF_OK, CWTHF_E_BAD_INPUT (negative / NaN)
// or CWTHF_E_OVERFLOW (>= 2^31).
__device__ __forceinline__ int mass_quantum(const DepArgs& a, int64_t i, uint32_t& mq) {
    mq = 0;
    if (!a.mass) { mq = 1; return CWTHF_OK; }
    float m = a.mass[i];
    if (!(m >= 0.0f)) return CWTHF_E_BAD_INPUT;
    double r = rint(__ddiv_rn(double(m), a.mass_unit));
    if (!(r < 2147483648.0)) return CWTHF_E_OVERFLOW;
    mq = uint32_t(r);
    return CWTHF_OK;
}

}  // namespace cwthf
