// quant.cuh -- the fixed-point position and mass rules shared by the deposit
// and the particle assignment (one definition, so both stages agree bit for bit).
#pragma once
#include "internal.cuh"

namespace cwthf {

struct DepArgs {
    const float* pos;
    const float* mass;
    double mass_unit;
    double scale;      // (ng / L) * 2^10, computed once on the host
    int64_t modulus;   // ng * 2^10
    int64_t np;
    int ng, ntx, nty, ntz;
};

inline DepArgs make_dep_args(const float* pos, const float* mass, double mass_unit, int64_t np, double L, int ng) {
    DepositGeom g = deposit_geom(ng);
    DepArgs a;
    a.pos = pos;
    a.mass = mass;
    a.mass_unit = mass_unit;
    a.scale = (double(ng) / L) * double(kFracOne);
    a.modulus = int64_t(ng) * kFracOne;
    a.np = np;
    a.ng = ng;
    a.ntx = g.ntx;
    a.nty = g.nty;
    a.ntz = g.ntz;
    return a;
}

// floor(x * scale) mod ng*2^10 with one correctly rounded fp64 product;
// false for non-finite or |x * scale| >= 2^40.
__device__ __forceinline__ bool quantise(float x, double scale, int64_t modulus, int64_t& q) {
    double t = __dmul_rn(double(x), scale);
    if (!(fabs(t) < 1099511627776.0)) return false;
    int64_t v = int64_t(floor(t)) % modulus;
    if (v < 0) v += modulus;
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
