// check.cuh -- opt-in bounds checks of the kernels' index arithmetic.
//
// Built with -DGBMC_CHECK (paper_1709_04394_gb300/build.py, check=True ->
// libgbmc_check.so), GBMC_IDX(i, n) verifies 0 <= i < n before an access: a
// failing index is recorded (the first failure's source line, per translation
// unit) and replaced by 0, so the access stays in bounds and the kernel goes
// on; the host reports the record at its next synchronising call
// (GBMC_ERR_STATE, "bounds check failed in <file>:<line>"). Without
// GBMC_CHECK, GBMC_IDX(i, n) is i and costs nothing. This is the library's
// stand-in for a memory checker: it is meant for small and uneven test
// lattices, not for timing.
#pragma once
#include <cstdint>

#ifdef GBMC_CHECK
#include <cuda_runtime.h>

namespace gbmc {

// Reads and clears one translation unit's record: true and the line if a check failed.
using CheckReader = bool (*)(unsigned* line);
void check_register(CheckReader reader, const char* file);

namespace {

__device__ unsigned int g_check_record[2];  // [0]: a check failed, [1]: its line

bool read_check_record(unsigned* line) {
    unsigned h[2] = {0u, 0u};
    if (cudaMemcpyFromSymbol(h, g_check_record, sizeof(h)) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (!h[0]) return false;
    const unsigned z[2] = {0u, 0u};
    cudaMemcpyToSymbol(g_check_record, z, sizeof(z));
    *line = h[1];
    return true;
}

struct CheckRegistrar {
    CheckRegistrar() { check_register(read_check_record, __BASE_FILE__); }
};
CheckRegistrar g_check_registrar;

__device__ __forceinline__ uint64_t check_index(uint64_t i, uint64_t n, unsigned line) {
    if (i < n) return i;
    if (atomicCAS(&g_check_record[0], 0u, 1u) == 0u) g_check_record[1] = line;
    return 0;
}

}  // namespace
}  // namespace gbmc

#define GBMC_IDX(i, n) (::gbmc::check_index((uint64_t)(i), (uint64_t)(n), __LINE__))
#else
#define GBMC_IDX(i, n) (i)
#endif
