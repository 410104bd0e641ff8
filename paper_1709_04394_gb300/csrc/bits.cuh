// bits.cuh -- bit-sliced updates of 32 same-colour sites held in one word
// (one bit per spin, 1 = down): int8 <-> bit conversion, acceptance bits and
// the word updates shared by the bit-packed layout (bitpack.cu), the
// bit-sliced resident sweeps (bitsweep.cu) and the bit-sliced double
// checkerboard (dcb_bits.cu).
#pragma once
#include <cstdint>

#include "device.cuh"

namespace gbmc {

// Down bits of the four bytes (+1 = 0x01, -1 = 0xFF) of a word: bit i = byte i
// is negative (the four sign bits gathered by one multiply).
__device__ __forceinline__ uint32_t nib_down(uint32_t four_bytes) {
    return ((four_bytes & 0x80808080u) * 0x00204081u) >> 28;
}

// Four down bits -> four bytes +1 / -1 (bit i to byte i, then 0 -> 0x01, 1 -> 0xFF).
__device__ __forceinline__ uint32_t spread4(uint32_t n) {
    return ((n * 0x00204081u) & 0x01010101u) * 0xFEu + 0x01010101u;
}

// Eight consecutive sites (bytes b0..b7 in lo, hi) -> the down bits of the four
// even-x sites (b0, b2, b4, b6) and of the four odd-x sites.
__device__ __forceinline__ void pack8(uint32_t lo, uint32_t hi, uint32_t& ev, uint32_t& od) {
    ev = nib_down(__byte_perm(lo, hi, 0x6420));
    od = nib_down(__byte_perm(lo, hi, 0x7531));
}

// The inverse: four even-x and four odd-x down bits -> eight bytes.
__device__ __forceinline__ uint2 unpack8(uint32_t ev, uint32_t od) {
    const uint32_t e = spread4(ev), o = spread4(od);
    return make_uint2(__byte_perm(e, o, 0x5140), __byte_perm(e, o, 0x7362));
}

// r4 = 2 r4 + [u <= T4], r8 = 2 r8 + [u <= T8]: the carry of T - u (set iff
// no borrow, i.e. u <= T) shifted in by an add-with-carry, two instructions
// per comparison. After 32 calls the first word's bit is bit 31 (__brev puts
// it back at bit 0).
__device__ __forceinline__ void accept_bits(uint32_t& r4, uint32_t& r8, uint32_t T4, uint32_t T8, uint32_t u) {
    asm("{\n\t.reg .u32 t;\n\t"
        "sub.cc.u32 t, %2, %4;\n\t"
        "addc.u32 %0, %0, %0;\n\t"
        "sub.cc.u32 t, %3, %4;\n\t"
        "addc.u32 %1, %1, %1;\n\t}"
        : "+r"(r4), "+r"(r8)
        : "r"(T4), "r"(T8), "r"(u));
}

// Philox4x32-10 of philox_q (device.cuh) with each 32 x 32 -> 64-bit product
// as one wide multiply (both halves from one instruction): the same words,
// fewer multiply-pipe instructions in the bit-sliced updates, where the
// products dominate that pipe.
__device__ __forceinline__ void mulhilo_wide(uint32_t a, uint32_t b, uint32_t& hi, uint32_t& lo) {
    uint64_t p;
    asm("mul.wide.u32 %0, %1, %2;" : "=l"(p) : "r"(a), "r"(b));
    hi = (uint32_t)(p >> 32);
    lo = (uint32_t)p;
}

__device__ __forceinline__ uint4 philox_q_wide(const PhiloxFixed& f, uint32_t q) {
    uint32_t x, y;
    mulhilo_wide(kPhiloxM0, q, x, y);
    x ^= f.x0;
    uint32_t h1, l1;
    mulhilo_wide(kPhiloxM1, x, h1, l1);
    uint4 c = make_uint4(h1 ^ f.b1, l1, f.u1 ^ y, f.v1);
    uint32_t k0 = f.k0, k1 = f.k1;
#pragma unroll
    for (int round = 2; round < 10; ++round) {
        uint32_t hi0, lo0, hi1, lo1;
        mulhilo_wide(kPhiloxM0, c.x, hi0, lo0);
        mulhilo_wide(kPhiloxM1, c.z, hi1, lo1);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += kPhiloxW0;
        k1 += kPhiloxW1;
    }
    return c;
}

// r = 2 r + [u <= T]: one comparison.
__device__ __forceinline__ void accept_bit(uint32_t& r, uint32_t T, uint32_t u) {
    asm("{\n\t.reg .u32 t;\n\t"
        "sub.cc.u32 t, %1, %2;\n\t"
        "addc.u32 %0, %0, %0;\n\t}"
        : "+r"(r)
        : "r"(T), "r"(u));
}

// r4, r8, r12 shifted by one bit each: three comparisons of u (3D, dE = 4,
// 8, 12).
__device__ __forceinline__ void accept_bits3(uint32_t& r4, uint32_t& r8, uint32_t& r12, uint32_t T4, uint32_t T8,
                                             uint32_t T12, uint32_t u) {
    accept_bits(r4, r8, T4, T8, u);
    asm("{\n\t.reg .u32 t;\n\t"
        "sub.cc.u32 t, %1, %2;\n\t"
        "addc.u32 %0, %0, %0;\n\t}"
        : "+r"(r12)
        : "r"(T12), "r"(u));
}

// The new value of the word s (32 sites of one colour) given its neighbour
// words; q0 = the Philox counter q of its first site (colour rank k = y L/2 +
// 32 w + b of bit b, q = k / 4).
__device__ __forceinline__ uint32_t bp_word_update(uint32_t s, uint32_t up, uint32_t dn, uint32_t same, uint32_t side,
                                                   const PhiloxFixed& pf, uint32_t q0, uint32_t T4, uint32_t T8) {
    const uint32_t d1 = s ^ up, d2 = s ^ dn, d3 = s ^ same, d4 = s ^ side;  // 1 = unsatisfied bond
    // bit-sliced a = d1 + d2 + d3 + d4 = a0 + 2 a1 + 4 a2
    const uint32_t s1 = d1 ^ d2, c1 = d1 & d2, s2 = d3 ^ d4, c2 = d3 & d4;
    const uint32_t a0 = s1 ^ s2, c3 = s1 & s2;
    const uint32_t a1 = c1 ^ c2 ^ c3, a2 = (c1 & c2) | (c3 & (c1 ^ c2));
    const uint32_t ge2 = a1 | a2;            // dE <= 0: always flips
    const uint32_t eq1 = a0 & ~ge2;          // dE = 4
    const uint32_t eq0 = ~(a0 | ge2);        // dE = 8
    uint32_t r4 = 0, r8 = 0;                 // bit b of the word at bit 31 - b
#pragma unroll
    for (uint32_t i = 0; i < 8; ++i) {
        const uint4 v = philox_q_wide(pf, q0 + i);
        accept_bits(r4, r8, T4, T8, v.x);
        accept_bits(r4, r8, T4, T8, v.y);
        accept_bits(r4, r8, T4, T8, v.z);
        accept_bits(r4, r8, T4, T8, v.w);
    }
    return s ^ (ge2 | (eq1 & __brev(r4)) | (eq0 & __brev(r8)));
}

// Majority of three words, bit by bit (the carry of a full adder).
__device__ __forceinline__ uint32_t maj3(uint32_t a, uint32_t b, uint32_t c) { return (a & b) | (c & (a ^ b)); }

// 3D: the new value of the word s given its six unsatisfied-bond masks d0..d5
// (bit = 1 where s_i J_ij s_j = -1). a = d0 + .. + d5 bit-sliced; a site flips
// iff a >= 3 (dE <= 0), or a = 2 and u <= T(4), a = 1 and u <= T(8), a = 0 and
// u <= T(12). q0: Philox counter q of the word's first site.
__device__ __forceinline__ uint32_t bp3_word_update(uint32_t s, uint32_t d0, uint32_t d1, uint32_t d2, uint32_t d3,
                                                    uint32_t d4, uint32_t d5, const PhiloxFixed& pf, uint32_t q0,
                                                    uint32_t T4, uint32_t T8, uint32_t T12) {
    const uint32_t s1 = d0 ^ d1 ^ d2, c1 = maj3(d0, d1, d2);
    const uint32_t s2 = d3 ^ d4 ^ d5, c2 = maj3(d3, d4, d5);
    const uint32_t a0 = s1 ^ s2, t = s1 & s2;
    const uint32_t a1 = c1 ^ c2 ^ t, a2 = maj3(c1, c2, t);
    const uint32_t ge3 = a2 | (a1 & a0);     // dE <= 0
    const uint32_t eq2 = a1 & ~(a0 | a2);    // dE = 4
    const uint32_t eq1 = a0 & ~(a1 | a2);    // dE = 8
    const uint32_t eq0 = ~(a0 | a1 | a2);    // dE = 12
    uint32_t r4 = 0, r8 = 0, r12 = 0;
#pragma unroll
    for (uint32_t i = 0; i < 8; ++i) {
        const uint4 v = philox_q_wide(pf, q0 + i);
        accept_bits3(r4, r8, r12, T4, T8, T12, v.x);
        accept_bits3(r4, r8, r12, T4, T8, T12, v.y);
        accept_bits3(r4, r8, r12, T4, T8, T12, v.z);
        accept_bits3(r4, r8, r12, T4, T8, T12, v.w);
    }
    return s ^ (ge3 | (eq2 & __brev(r4)) | (eq1 & __brev(r8)) | (eq0 & __brev(r12)));
}

}  // namespace gbmc
