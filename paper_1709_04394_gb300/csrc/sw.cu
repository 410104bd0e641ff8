// sw.cu -- Swendsen-Wang cluster updates of the Ising ferromagnet (Sec. 3.3):
// bond activation, connected components, cluster flips.
//
//  k_sw_bonds : one thread per 4 sites. Forward bond b = dim i + mu is active
//               iff s_i = s_j and its Philox word (purpose 6, counter
//               (b >> 2, t, replica, c3), word b & 3) is <= T_bond =
//               ceil((1 - exp(-2 beta)) 2^32) - 1; bit mu of bonds[i]. Also
//               resets parent[i] = i.
//  k_sw_union : one thread per site unites i with the far end of each of its
//               active bonds in a lock-free union-find (atomicMin hooks the
//               larger root under the smaller one; a hook that lost a race
//               retries from the value it found, so no link is dropped). Every
//               component ends as one tree rooted at its smallest site.
//  k_sw_flip  : one thread per site finds its root r (with path halving) and
//               flips iff the top bit of r's Philox word (purpose 7, counter
//               (r >> 2, t, replica, c3), word r & 3) is 1; optionally writes r.
// Parent pointers only ever decrease, so every find walks a strictly
// decreasing chain and ends; the hook loops are additionally capped (error flag).
//
// Tiled labelling (2D L % 32 == 0: 32 x 32 tiles; 3D L % 16 == 0: 16 x 8 x 8),
// the tile decomposition of Sec. 3.3 with the consolidation done by atomics:
//  k_sw_local : one CTA per tile computes the tile's bond flags (the same
//               Philox words as k_sw_bonds), labels the tile's components in
//               shared memory with the same lock-free union-find, and writes
//               parent[i] = the smallest site of i's component within the
//               tile (global index: increasing with the local one);
//  k_sw_cross : the bonds that leave a tile are united in the global forest.
// Each component again ends rooted at its smallest site.
#include "device.cuh"
#include "internal.h"

namespace gbmc {

constexpr uint32_t kPurposeSwBond = 6u, kPurposeSwFlip = 7u;
constexpr uint32_t kSwHookCap = 1u << 24;

__device__ __forceinline__ uint32_t sw_forward(uint32_t i, uint32_t mu, uint32_t L, uint32_t dim) {
    const uint32_t x = i % L, y = (i / L) % L;
    if (mu == 0) return i - x + (x + 1 == L ? 0 : x + 1);
    if (mu == 1) return i + (y + 1 == L ? 0 - (L - 1) * L : L);
    const uint32_t LL = L * L, z = i / LL;
    return i + (z + 1 == L ? 0 - (L - 1) * LL : LL);
}

// Forest reads: global forests through L2 (other CTAs hook concurrently),
// shared-memory forests through volatile loads.
template <bool GLOBAL>
__device__ __forceinline__ uint32_t sw_ld(uint32_t* p) {
    if constexpr (GLOBAL) return __ldcg(p);
    else return *reinterpret_cast<volatile uint32_t*>(p);
}

template <bool GLOBAL>
__device__ __forceinline__ uint32_t sw_find(uint32_t* par, uint32_t x) {
    uint32_t cur = sw_ld<GLOBAL>(par + x);
    if (cur == x) return x;
    uint32_t prev = x, next;
    while (cur > (next = sw_ld<GLOBAL>(par + cur))) {
        par[prev] = next;  // path halving: pointers only move to smaller indices
        prev = cur;
        cur = next;
    }
    return cur;
}

// The active flags (bit mu) of the forward bonds of sites i0 .. i0 + 3
// (i0 % 4 == 0): dim Philox calls cover bonds dim i0 .. dim (i0 + 4) - 1.
__device__ __forceinline__ void sw_bond_flags(const SwLaunch& P, const int8_t* s, uint32_t i0, uint32_t r,
                                              uint32_t c3, uint32_t flags[4]) {
    flags[0] = flags[1] = flags[2] = flags[3] = 0u;
    for (uint32_t c = 0; c < P.dim; ++c) {
        const uint32_t q = (P.dim * i0) / 4 + c;
        const uint4 w = philox4x32_10(make_uint4(q, P.t, r, c3), (uint32_t)P.seed, (uint32_t)(P.seed >> 32));
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t b = 4 * q + k, i = b / P.dim, mu = b - i * P.dim;
            const uint32_t u = k == 0 ? w.x : k == 1 ? w.y : k == 2 ? w.z : w.w;
            const uint32_t j = sw_forward(i, mu, P.L, P.dim);
            if (s[i] == s[j] && (long long)u <= P.T_bond) flags[i - i0] |= 1u << mu;
        }
    }
}

// Lock-free union of a and b in forest par (global or shared memory).
template <bool GLOBAL>
__device__ __forceinline__ void sw_unite(uint32_t* par, uint32_t a, uint32_t b, unsigned int* err) {
    uint32_t ra = sw_find<GLOBAL>(par, a), rb = sw_find<GLOBAL>(par, b);
    uint32_t n = 0;
    while (ra != rb) {
        if (ra > rb) {
            const uint32_t tmp = ra;
            ra = rb;
            rb = tmp;
        }
        const uint32_t old = atomicMin(par + rb, ra);  // hook the larger root under the smaller
        if (old == rb) break;
        rb = sw_find<GLOBAL>(par, old);  // rb had been hooked meanwhile: merge with its new root
        ra = sw_find<GLOBAL>(par, ra);
        if (++n == kSwHookCap) {
            atomicExch(err, 1u);
            break;
        }
    }
}

__global__ void __launch_bounds__(256) k_sw_bonds(const __grid_constant__ SwLaunch P) {
    const uint64_t copy = P.copy0 + blockIdx.y;
    const uint32_t i0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (i0 >= P.N) return;
    const int8_t* s = P.spins + copy * P.N;
    uint8_t* bonds = P.bonds + copy * P.N;
    uint32_t* par = P.parent + copy * P.N;
    const uint32_t inst = (uint32_t)(copy / P.R), r = (uint32_t)(copy - (uint64_t)inst * P.R);
    const uint32_t c3 = c3_word(kPurposeSwBond, 0u, P.inst_base + inst);
    uint32_t flags[4];
    sw_bond_flags(P, s, i0, r, c3, flags);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        bonds[i0 + k] = (uint8_t)flags[k];
        par[i0 + k] = i0 + k;
    }
}

struct SwTile {
    uint32_t tx, ty, tz;  // tile edge lengths
};

__device__ __forceinline__ SwTile sw_tile(uint32_t dim) {
    return dim == 2 ? SwTile{32u, 32u, 1u} : SwTile{16u, 8u, 8u};
}

__global__ void __launch_bounds__(256) k_sw_local(const __grid_constant__ SwLaunch P) {
    __shared__ uint32_t lp[1024];
    const uint64_t copy = P.copy0 + blockIdx.y;
    const int8_t* s = P.spins + copy * P.N;
    const uint32_t inst = (uint32_t)(copy / P.R), r = (uint32_t)(copy - (uint64_t)inst * P.R);
    const uint32_t c3 = c3_word(kPurposeSwBond, 0u, P.inst_base + inst);
    const SwTile T = sw_tile(P.dim);
    const uint32_t ntx = P.L / T.tx, nty = P.L / T.ty;
    const uint32_t bx = blockIdx.x % ntx, by = (blockIdx.x / ntx) % nty, bz = blockIdx.x / (ntx * nty);
    // thread t: local sites l = 4t .. 4t+3 (consecutive x in one tile row)
    const uint32_t l0 = 4 * threadIdx.x;
    const uint32_t lx = l0 % T.tx, ly = (l0 / T.tx) % T.ty, lz = l0 / (T.tx * T.ty);
    const uint32_t i0 = ((bz * T.tz + lz) * P.L + by * T.ty + ly) * P.L + bx * T.tx + lx;
    uint32_t flags[4];
    sw_bond_flags(P, s, i0, r, c3, flags);
#pragma unroll
    for (int k = 0; k < 4; ++k) lp[l0 + k] = l0 + k;
    __syncthreads();
    // bonds inside the tile: unite in shared memory
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint32_t l = l0 + k, x = lx + k;
        if ((flags[k] & 1u) && x + 1 < T.tx) sw_unite<false>(lp, l, l + 1, P.err);
        if ((flags[k] & 2u) && ly + 1 < T.ty) sw_unite<false>(lp, l, l + T.tx, P.err);
        if ((flags[k] & 4u) && lz + 1 < T.tz) sw_unite<false>(lp, l, l + T.tx * T.ty, P.err);
    }
    __syncthreads();
    uint32_t* par = P.parent + copy * P.N;
    uint8_t* bonds = P.bonds + copy * P.N;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint32_t root = sw_find<false>(lp, l0 + k);
        const uint32_t rx = root % T.tx, ry = (root / T.tx) % T.ty, rz = root / (T.tx * T.ty);
        par[i0 + k] = ((bz * T.tz + rz) * P.L + by * T.ty + ry) * P.L + bx * T.tx + rx;
        bonds[i0 + k] = (uint8_t)flags[k];
    }
}

// Bonds that leave their tile, united in the global forest.
__global__ void __launch_bounds__(256) k_sw_cross(const __grid_constant__ SwLaunch P) {
    const uint64_t copy = P.copy0 + blockIdx.y;
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.N) return;
    const uint8_t f = P.bonds[copy * P.N + i];
    if (!f) return;
    const SwTile T = sw_tile(P.dim);
    const uint32_t x = i % P.L, y = (i / P.L) % P.L, z = i / (P.L * P.L);
    uint32_t* par = P.parent + copy * P.N;
    if ((f & 1u) && x % T.tx == T.tx - 1) sw_unite<true>(par, i, sw_forward(i, 0, P.L, P.dim), P.err);
    if ((f & 2u) && y % T.ty == T.ty - 1) sw_unite<true>(par, i, sw_forward(i, 1, P.L, P.dim), P.err);
    if ((f & 4u) && z % T.tz == T.tz - 1) sw_unite<true>(par, i, sw_forward(i, 2, P.L, P.dim), P.err);
}

__global__ void __launch_bounds__(256) k_sw_union(const __grid_constant__ SwLaunch P) {
    const uint64_t copy = P.copy0 + blockIdx.y;
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.N) return;
    const uint8_t f = P.bonds[copy * P.N + i];
    if (!f) return;
    uint32_t* par = P.parent + copy * P.N;
    for (uint32_t mu = 0; mu < P.dim; ++mu)
        if ((f >> mu) & 1u) sw_unite<true>(par, i, sw_forward(i, mu, P.L, P.dim), P.err);
}

__global__ void __launch_bounds__(256) k_sw_flip(const __grid_constant__ SwLaunch P) {
    const uint64_t copy = P.copy0 + blockIdx.y;
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.N) return;
    uint32_t* par = P.parent + copy * P.N;
    const uint32_t root = sw_find<true>(par, i);
    const uint32_t inst = (uint32_t)(copy / P.R), r = (uint32_t)(copy - (uint64_t)inst * P.R);
    const uint4 w = philox4x32_10(make_uint4(root >> 2, P.t, r, c3_word(kPurposeSwFlip, 0u, P.inst_base + inst)),
                                  (uint32_t)P.seed, (uint32_t)(P.seed >> 32));
    const uint32_t word = (root & 3u) == 0 ? w.x : (root & 3u) == 1 ? w.y : (root & 3u) == 2 ? w.z : w.w;
    if (word >> 31) P.spins[copy * P.N + i] = (int8_t)(-P.spins[copy * P.N + i]);
    if (P.labels) P.labels[copy * P.N + i] = (int32_t)root;
}

cudaError_t launch_sw_update(const SwLaunch& P0, uint64_t copies, cudaStream_t s) {
    if (P0.N % 4 != 0) return cudaErrorInvalidValue;
    for (uint64_t c0 = 0; c0 < copies; c0 += 65535) {
        SwLaunch P = P0;
        P.copy0 = c0;
        const uint32_t nc = (uint32_t)((copies - c0) < 65535 ? (copies - c0) : 65535);
        const uint32_t quads = P.N / 4;
        const bool tiled = (P.dim == 2 && P.L % 32 == 0) || (P.dim == 3 && P.L % 16 == 0);
        cudaError_t e;
        if (tiled) {
            k_sw_local<<<dim3(P.N / 1024, nc), 256, 0, s>>>(P);
            count_launch();
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            k_sw_cross<<<dim3((P.N + 255) / 256, nc), 256, 0, s>>>(P);
            count_launch();
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        } else {
            k_sw_bonds<<<dim3((quads + 255) / 256, nc), 256, 0, s>>>(P);
            count_launch();
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            k_sw_union<<<dim3((P.N + 255) / 256, nc), 256, 0, s>>>(P);
            count_launch();
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        k_sw_flip<<<dim3((P.N + 255) / 256, nc), 256, 0, s>>>(P);
        count_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace gbmc
