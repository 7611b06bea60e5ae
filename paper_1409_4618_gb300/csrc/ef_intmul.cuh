// FP64 multiplication on the integer pipes, bit for bit what the FP64
// multiply instruction gives (IEEE 754 binary64, round to nearest, ties to
// even), for use beside the FP64 pipe in the element kernels.
//
// On this GPU the FP64 pipe retires at most 2 lane operations per SM per
// clock (1.68 for DMUL), while the integer ALU and IMAD pipes retire 64
// lanes each; the element kernels keep the FP64 pipe busy and leave the
// integer pipes nearly idle. A product computed here takes about 50 integer
// instructions (ALU and IMAD) and runs beside the FP64 instructions of the
// same warps, so moving the products of an element routine here shortens its
// critical resource by their share.
//
// Method (the textbook one for a binary floating-point product, e.g.
// J.-M. Muller et al., Handbook of Floating-Point Arithmetic, 2nd ed., Sec.
// 7.4): the 53-bit significands with their hidden bits, split into 21- and
// 32-bit limbs, give the exact 106-bit product from three 32x32->64-bit
// multiplies (one of them with a 64-bit addend). It lies in [2^104, 2^106), so
// its leading 53 bits start at bit 105 or 104 (top); below them the next bit
// (round) and the OR of all lower bits (sticky) decide the rounding to nearest,
// ties to even: add one to the 53 bits if round is set and sticky or their
// last bit is. The exponent field is added to the significand (hidden bit
// included, hence the field minus one), so a carry out of the significand
// steps the exponent.
//
// Zero operands give a signed zero here. Subnormal, infinite or NaN operands,
// and results that would overflow or leave the normal range, set `off`; the
// caller then repeats the element with the FP64 instruction (FpMul), so that
// every element gets exactly the bits of the routine with FP64 products.
#pragma once

#include <stdint.h>

namespace ef {

// The bit pattern of a double and back, through an opaque move: written as
// plain bit casts, tests on the pattern (zero, exponent range) are turned by
// the compiler into FP64 comparisons, which run on the FP64 pipe (measured:
// about one per distinct operand in the 3D Nedelec element routine).
__device__ __forceinline__ uint64_t bits_of(double x)
{
    uint64_t b;
    asm("mov.b64 %0, %1;" : "=l"(b) : "d"(x));
    return b;
}

__device__ __forceinline__ double double_of(uint64_t b)
{
    double x;
    asm("mov.b64 %0, %1;" : "=d"(x) : "l"(b));
    return x;
}

struct IntMul {
    uint32_t off = 0;
    __device__ __forceinline__ double operator()(double a, double b)
    {
        const uint64_t ua = bits_of(a), ub = bits_of(b);
        const uint32_t ahi = (uint32_t)(ua >> 32), alo = (uint32_t)ua, bhi = (uint32_t)(ub >> 32), blo = (uint32_t)ub;
        const uint32_t ea = (ahi >> 20) & 0x7ffu, eb = (bhi >> 20) & 0x7ffu;
        // significands a1 2^32 + a0, b1 2^32 + b0 with the hidden bit (a1, b1 < 2^21)
        const uint32_t a1 = (ahi & 0xfffffu) | 0x100000u, b1 = (bhi & 0xfffffu) | 0x100000u;
        // exact product P = w23 2^64 + w1 2^32 + w0 in [2^104, 2^106)
        const uint64_t t0 = (uint64_t)alo * blo;
        const uint64_t m = (uint64_t)a1 * blo + (uint64_t)alo * b1;   // < 2^54
        const uint64_t w1x = (t0 >> 32) + (uint32_t)m;
        const uint32_t w0 = (uint32_t)t0, w1 = (uint32_t)w1x;
        const uint64_t w23 = (uint64_t)a1 * b1 + (m >> 32) + (w1x >> 32);   // < 2^42
        // 53 result bits: P >> (52 + top), top = bit 105 of P
        const uint32_t top = (uint32_t)(w23 >> 41);
        const uint32_t sh = 20u + top;
        const uint32_t qlo = __funnelshift_r(w1, (uint32_t)w23, sh);
        const uint32_t qhi = (uint32_t)(w23 >> sh);
        const uint32_t rnd = (w1 >> (sh - 1u)) & 1u;
        const uint32_t sticky = ((w1 & ((1u << (sh - 1u)) - 1u)) | w0) != 0u;
        const uint32_t inc = rnd & (sticky | (qlo & 1u));
        const int E1 = (int)ea + (int)eb - 1024 + (int)top;   // result exponent field minus one
        const uint64_t sign = (uint64_t)((ahi ^ bhi) & 0x80000000u) << 32;
        uint64_t r = ((((uint64_t)qhi << 32) | qlo) + inc + ((uint64_t)(uint32_t)E1 << 52)) | sign;
        const bool zero = ((ahi & 0x7fffffffu) | alo) == 0u || ((bhi & 0x7fffffffu) | blo) == 0u;
        r = zero ? sign : r;
        off |= (uint32_t)((ea == 0x7ffu) | (eb == 0x7ffu) |
                          (!zero & ((ea == 0u) | (eb == 0u) | ((uint32_t)E1 > 0x7fdu))));
        return double_of(r);
    }
};

// The FP64 instruction, for the repeat of an element that IntMul flagged and
// for kernels that keep their products on the FP64 pipe; __dmul_rn is never
// contracted into an FMA with a following addition, as an IntMul product
// cannot be either, so both give the same bits.
struct FpMul {
    uint32_t off = 0;
    __device__ __forceinline__ double operator()(double a, double b) { return __dmul_rn(a, b); }
};

}  // namespace ef
