// device.cuh -- device-side building blocks shared by the library's kernels:
// the Philox4x32-10 counter-based generator (Sec. 4) and warp/block reductions.
#pragma once
#include <cstdint>

namespace gbmc {

// Philox4x32-10 (Salmon et al. 2011, as summarised in Sec. 4): ten rounds of
// (L, R) -> (mullo(R, M), mulhi(R, M) ^ k ^ L) on the two word pairs with the
// 4x32 permutation, key advanced by the Weyl increments between rounds.
constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

enum : uint32_t { kPurposeMetro = 0u, kPurposeInit = 1u, kPurposeResample = 2u, kPurposeCoupling = 3u };

// 32 x 32 -> 64-bit product as (hi, lo). Two 32-bit multiplies (high and low
// half) measured faster on sm_103a than one 64-bit product.
__device__ __forceinline__ void mulhilo(uint32_t a, uint32_t b, uint32_t& hi, uint32_t& lo) {
    hi = __umulhi(a, b);
    lo = a * b;
}

__device__ __forceinline__ uint32_t c3_word(uint32_t purpose, uint32_t colour, uint32_t instance) {
    return (purpose << 28) | (colour << 27) | instance;
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        uint32_t hi0, lo0, hi1, lo1;
        mulhilo(kPhiloxM0, c.x, hi0, lo0);
        mulhilo(kPhiloxM1, c.z, hi1, lo1);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += kPhiloxW0;
        k1 += kPhiloxW1;
    }
    return c;
}

// Same result as philox4x32_10((q, t, r, c3), k0, k1) for callers whose t, r
// and c3 stay fixed over many values of q: round 0's product of r, and round
// 1's product of the (q-independent) first word, are hoisted into
// PhiloxFixed, leaving 18 of the 20 wide products per call.
struct PhiloxFixed {
    uint32_t x0;   // round 0, word 2 before the q-dependent mulhi: c3 ^ k1
    uint32_t b1;   // round 1, word 0 before the q-dependent mulhi: lo(M1 r) ^ (k0 + W0)
    uint32_t u1;   // round 1, word 2 before the q-dependent xor: hi(M0 A) ^ (k1 + W1)
    uint32_t v1;   // round 1, word 3: lo(M0 A), A = hi(M1 r) ^ t ^ k0
    uint32_t k0, k1;  // key of round 2
};

__device__ __forceinline__ PhiloxFixed philox_fix(uint32_t t, uint32_t r, uint32_t c3, uint32_t k0,
                                                  uint32_t k1) {
    PhiloxFixed f;
    const uint32_t a = __umulhi(kPhiloxM1, r) ^ t ^ k0;
    const uint32_t b = kPhiloxM1 * r;
    f.x0 = c3 ^ k1;
    f.b1 = b ^ (k0 + kPhiloxW0);
    f.u1 = __umulhi(kPhiloxM0, a) ^ (k1 + kPhiloxW1);
    f.v1 = kPhiloxM0 * a;
    f.k0 = k0 + 2u * kPhiloxW0;
    f.k1 = k1 + 2u * kPhiloxW1;
    return f;
}

__device__ __forceinline__ uint4 philox_q(const PhiloxFixed& f, uint32_t q) {
    // round 0: words 2, 3 depend on q
    uint32_t x, y;
    mulhilo(kPhiloxM0, q, x, y);
    x ^= f.x0;
    // round 1
    uint32_t h1, l1;
    mulhilo(kPhiloxM1, x, h1, l1);
    uint4 c = make_uint4(h1 ^ f.b1, l1, f.u1 ^ y, f.v1);
    uint32_t k0 = f.k0, k1 = f.k1;
#pragma unroll
    for (int round = 2; round < 10; ++round) {
        uint32_t hi0, lo0, hi1, lo1;
        mulhilo(kPhiloxM0, c.x, hi0, lo0);
        mulhilo(kPhiloxM1, c.z, hi1, lo1);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += kPhiloxW0;
        k1 += kPhiloxW1;
    }
    return c;
}

__device__ __forceinline__ uint32_t word_of(const uint4& w, uint32_t lane) {
    return lane == 0 ? w.x : lane == 1 ? w.y : lane == 2 ? w.z : w.w;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Inclusive scan across a warp.
template <typename T>
__device__ __forceinline__ T warp_inclusive_scan(T v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T n = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += n;
    }
    return v;
}

// Inclusive scan across the block (blockDim.x a multiple of 32, <= 1024).
// `shared` must hold 32 elements. Returns the inclusive prefix; *total gets the
// block total. Contains __syncthreads(): call from every thread.
template <typename T>
__device__ __forceinline__ T block_inclusive_scan(T v, T* shared, T* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    T x = warp_inclusive_scan(v);
    if (lane == 31) shared[warp] = x;
    __syncthreads();
    if (warp == 0) {
        T s = lane < nwarps ? shared[lane] : T(0);
        s = warp_inclusive_scan(s);
        if (lane < nwarps) shared[lane] = s;
    }
    __syncthreads();
    if (warp > 0) x += shared[warp - 1];
    if (total) *total = shared[nwarps - 1];
    __syncthreads();
    return x;
}

}  // namespace gbmc
