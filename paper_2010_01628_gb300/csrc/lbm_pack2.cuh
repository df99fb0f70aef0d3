// lbm_pack2.cuh -- two FP32 lanes in one register pair, computed with the
// packed FP32x2 instructions of sm_100+ (add/sub/mul/fma .f32x2): one issue
// slot updates two lattice nodes.  Each component is rounded exactly like the
// scalar FP32 operation (round to nearest even, no flush to zero).
//
// P2 plugs into the collision templates written for a scalar C: it converts
// from constants (broadcast), and a product a * b stays unevaluated (P2Mul)
// until it is added, subtracted or stored, so a * b + c issues one packed fma
// as the scalar compiler's contraction would.
#pragma once

#include <cuda_runtime.h>

namespace lbm {

__device__ __forceinline__ unsigned long long p2_bits(float2 a) {
    return (unsigned long long)__float_as_uint(a.x) | ((unsigned long long)__float_as_uint(a.y) << 32);
}
__device__ __forceinline__ float2 p2_from_bits(unsigned long long r) {
    return make_float2(__uint_as_float((unsigned)r), __uint_as_float((unsigned)(r >> 32)));
}
__device__ __forceinline__ float2 p2_sub(float2 a, float2 b) {
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(p2_bits(a)), "l"(p2_bits(b)));
    return p2_from_bits(d);
}
// Sign flip of both lanes by an integer XOR: the ALU pipe does it, leaving the
// FP32 pipe (which the packed collision keeps busy) to the arithmetic.
__device__ __forceinline__ float2 p2_neg(float2 a) {
    return make_float2(__uint_as_float(__float_as_uint(a.x) ^ 0x80000000u),
                       __uint_as_float(__float_as_uint(a.y) ^ 0x80000000u));
}

struct P2 {
    float2 v;
    P2() = default;
    __device__ __forceinline__ P2(float2 a) : v(a) {}
    __device__ __forceinline__ P2(float a, float b) : v(make_float2(a, b)) {}
    __device__ __forceinline__ explicit P2(float s) : v(make_float2(s, s)) {}
    __device__ __forceinline__ explicit P2(double s) : P2((float)s) {}
    __device__ __forceinline__ explicit P2(int s) : P2((float)s) {}
    __device__ __forceinline__ P2& operator+=(P2 b);
    __device__ __forceinline__ P2& operator-=(P2 b);
    __device__ __forceinline__ P2& operator*=(P2 b);
};

// The product a * b, not yet rounded.
struct P2Mul {
    float2 a, b;
    __device__ __forceinline__ operator P2() const { return P2(__fmul2_rn(a, b)); }
};

__device__ __forceinline__ P2Mul operator*(P2 a, P2 b) { return P2Mul{a.v, b.v}; }
__device__ __forceinline__ P2Mul operator*(P2Mul p, P2 c) { return P2Mul{__fmul2_rn(p.a, p.b), c.v}; }
__device__ __forceinline__ P2Mul operator*(P2 c, P2Mul p) { return P2Mul{c.v, __fmul2_rn(p.a, p.b)}; }
__device__ __forceinline__ P2Mul operator*(P2Mul p, P2Mul q) { return P2Mul{__fmul2_rn(p.a, p.b), __fmul2_rn(q.a, q.b)}; }

__device__ __forceinline__ P2 operator+(P2 a, P2 b) { return P2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ P2 operator+(P2Mul p, P2 c) { return P2(__ffma2_rn(p.a, p.b, c.v)); }
__device__ __forceinline__ P2 operator+(P2 c, P2Mul p) { return P2(__ffma2_rn(p.a, p.b, c.v)); }
__device__ __forceinline__ P2 operator+(P2Mul p, P2Mul q) { return P2(__ffma2_rn(p.a, p.b, __fmul2_rn(q.a, q.b))); }

__device__ __forceinline__ P2 operator-(P2 a, P2 b) { return P2(p2_sub(a.v, b.v)); }
__device__ __forceinline__ P2 operator-(P2Mul p, P2 c) { return P2(__ffma2_rn(p.a, p.b, p2_neg(c.v))); }
__device__ __forceinline__ P2 operator-(P2 c, P2Mul p) { return P2(__ffma2_rn(p2_neg(p.a), p.b, c.v)); }
__device__ __forceinline__ P2 operator-(P2Mul p, P2Mul q) {
    return P2(__ffma2_rn(p.a, p.b, p2_neg(__fmul2_rn(q.a, q.b))));
}
__device__ __forceinline__ P2 operator-(P2 a) { return P2(p2_neg(a.v)); }
__device__ __forceinline__ P2Mul operator-(P2Mul p) { return P2Mul{p2_neg(p.a), p.b}; }

__device__ __forceinline__ P2& P2::operator+=(P2 b) { return *this = *this + b; }
__device__ __forceinline__ P2& P2::operator-=(P2 b) { return *this = *this - b; }
__device__ __forceinline__ P2& P2::operator*=(P2 b) { return *this = P2(__fmul2_rn(v, b.v)); }

// Reciprocal per lane by the hardware approximation (within about 1 ulp; the
// argument is a density near 1): the correctly rounded form costs a refinement
// and a special-case path on the FP32 pipe, which the 16-bit kernels are short
// of, for a difference far below their storage rounding.
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ P2 recip(P2 x) { return P2(rcp_approx(x.v.x), rcp_approx(x.v.y)); }

}  // namespace lbm
