// FP64 additions and constant multiples at the FP64 pipe's full rate.
//
// Measured on this GPU (ef_fp64_probe): a DFMA whose three operands are all
// per-thread registers retires 2 lane operations per SM per clock (0.63 T/s
// at 2,070 MHz); DADD, DMUL, and a DFMA with a literal constant or with a
// value the compiler knows to be the same in every thread (kept in a uniform
// register) retire 1.68 (84 %). So an addition here is a DFMA with a
// per-thread 1.0: fma(a, 1, b) rounds the exact a + b once, which is what
// DADD gives, bit for bit; a - b is fma(-b, 1, a); and the constant factors
// 2 and 3 of the element routines come from per-thread registers too. The
// registers hold values set from a thread index that the compiler cannot
// see through, so that it neither folds them into constants nor proves them
// uniform.
#pragma once

namespace ef {

// v in a per-thread register (the select is never taken the other way).
__device__ __forceinline__ double per_thread(double v)
{
    int t = threadIdx.x;
    asm volatile("" : "+r"(t));
    return t >= 0 ? v : 0.0;
}

struct FpK {
    double one, two, three;
    __device__ __forceinline__ FpK() : one(per_thread(1.0)), two(per_thread(2.0)), three(per_thread(3.0)) {}
    // a + b and a - b, bit for bit the FP64 addition
    __device__ __forceinline__ double add(double a, double b) const { return fma(a, one, b); }
    __device__ __forceinline__ double sub(double a, double b) const { return fma(-b, one, a); }
};

// The same operations with literal constants (DADD, DFMA with immediates):
// the same bits, three registers fewer, for kernels held to few registers.
struct FpLit {
    static constexpr double one = 1.0, two = 2.0, three = 3.0;
    __device__ __forceinline__ double add(double a, double b) const { return a + b; }
    __device__ __forceinline__ double sub(double a, double b) const { return a - b; }
};

}  // namespace ef
