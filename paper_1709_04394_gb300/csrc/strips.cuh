// strips.cuh -- the neighbour wait of strip-resident sweeps (a CTA keeps a
// strip of rows in shared memory for a whole call and trades its first and
// last rows with the CTAs of the strips above and below).
#pragma once
#include <cstdint>

namespace gbmc {

// Wait until both neighbours' progress counters reach `need` (they have
// published their boundary rows of that many half-sweeps). Bounded: gives up
// after `budget` cycles, or at once when *err is already raised, raising *err
// and returning false. Called by one thread per CTA or per warp, never by
// every thread (the polls are plain loads of two words).
__device__ __forceinline__ bool strip_wait(const unsigned int* pu, const unsigned int* pd, uint32_t need,
                                           unsigned int* err, long long budget) {
    const long long t0 = clock64();
    while (*reinterpret_cast<const volatile unsigned int*>(pu) < need ||
           *reinterpret_cast<const volatile unsigned int*>(pd) < need) {
        if (*reinterpret_cast<const volatile unsigned int*>(err) != 0u || clock64() - t0 > budget) {
            atomicExch(err, 1u);
            return false;
        }
        __nanosleep(32);
    }
    __threadfence();
    return true;
}

}  // namespace gbmc
