// bits.cuh -- acceptance bits of bit-parallel (multi-spin-coded) updates.
#pragma once
#include <cstdint>

namespace gbmc {

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

}  // namespace gbmc
