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
//  k_sw_local      : one CTA per tile computes the tile's bond flags (the same
//                    Philox words as k_sw_bonds), labels the tile's components
//                    in shared memory with the same lock-free union-find, and
//                    writes parent[i] = the smallest site of i's component
//                    within the tile (global index: increasing with the local one);
//  k_sw_cross      : one thread per bond that leaves a tile recomputes its
//                    flag and, if active, unites its ends in the global forest;
//  k_sw_flip_tiled : one CTA per tile copies the tile's parent pointers to
//                    shared memory and follows each site's chain there to the
//                    last node inside the tile; only those end nodes look up
//                    their root in the global forest and draw the root's coin,
//                    which every site of the tile then reads from shared memory.
// Each component again ends rooted at its smallest site (a hook always puts
// the larger root under the smaller), so the labels and coins do not depend
// on the order of the unions.
#include "bits.cuh"
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
// (i0 % 4 == 0): DIM Philox calls cover bonds DIM i0 .. DIM (i0 + 4) - 1; bond
// 4 c + k of them belongs to site i0 + (4 c + k) / DIM.
template <uint32_t DIM>
__device__ __forceinline__ void sw_bond_flags(const SwLaunch& P, const int8_t* s, uint32_t i0, uint32_t r,
                                              uint32_t c3, uint32_t flags[4]) {
    flags[0] = flags[1] = flags[2] = flags[3] = 0u;
#pragma unroll
    for (uint32_t c = 0; c < DIM; ++c) {
        const uint32_t q = (DIM * i0) / 4 + c;
        const uint4 w = philox4x32_10(make_uint4(q, P.t, r, c3), (uint32_t)P.seed, (uint32_t)(P.seed >> 32));
#pragma unroll
        for (uint32_t k = 0; k < 4; ++k) {
            const uint32_t n = (4 * c + k) / DIM, mu = (4 * c + k) % DIM, i = i0 + n;
            const uint32_t u = k == 0 ? w.x : k == 1 ? w.y : k == 2 ? w.z : w.w;
            const uint32_t j = sw_forward(i, mu, P.L, DIM);
            if (s[i] == s[j] && (long long)u <= P.T_bond) flags[n] |= 1u << mu;
        }
    }
}

// The same flags for sites i0 .. i0 + 3 = x0 .. x0 + 3 of row y, layer z
// (x0 % 4 == 0, so the four lie in one row): the spins come as 32-bit words
// (own, right-shifted by one site, row below, layer in front) and bit 1 of
// byte n of own ^ neighbour says whether site n differs from it (+-1 bytes).
template <uint32_t DIM>
__device__ __forceinline__ void sw_bond_flags_row(const SwLaunch& P, const int8_t* s, uint32_t i0, uint32_t x0,
                                                  uint32_t y, uint32_t z, uint32_t r, uint32_t c3,
                                                  uint32_t flags[4]) {
    const uint32_t L = P.L;
    const uint32_t own = *reinterpret_cast<const uint32_t*>(s + i0);
    const uint32_t nxt = (uint32_t)(uint8_t)s[i0 - x0 + (x0 + 4 == L ? 0 : x0 + 4)];
    uint32_t dif[DIM];
    dif[0] = own ^ ((own >> 8) | (nxt << 24));
    dif[1] = own ^ *reinterpret_cast<const uint32_t*>(s + (y + 1 == L ? i0 - (L - 1) * L : i0 + L));
    if constexpr (DIM == 3) {
        const uint32_t LL = L * L;
        dif[2] = own ^ *reinterpret_cast<const uint32_t*>(s + (z + 1 == L ? i0 - (L - 1) * LL : i0 + LL));
    }
    flags[0] = flags[1] = flags[2] = flags[3] = 0u;
    // the same words as philox4x32_10((q, t, r, c3)): t, r and c3 hoisted, wide products
    const PhiloxFixed pf = philox_fix(P.t, r, c3, (uint32_t)P.seed, (uint32_t)(P.seed >> 32));
#pragma unroll
    for (uint32_t c = 0; c < DIM; ++c) {
        const uint4 w = philox_q_wide(pf, (DIM * i0) / 4 + c);
#pragma unroll
        for (uint32_t k = 0; k < 4; ++k) {
            const uint32_t n = (4 * c + k) / DIM, mu = (4 * c + k) % DIM;
            const uint32_t u = k == 0 ? w.x : k == 1 ? w.y : k == 2 ? w.z : w.w;
            if (!((dif[mu] >> (8 * n + 1)) & 1u) && (long long)u <= P.T_bond) flags[n] |= 1u << mu;
        }
    }
}

// Whether forward bond mu of site i, to site j, is active: the same Philox
// word as in sw_bond_flags (bond b = dim i + mu, call b >> 2, word b & 3).
__device__ __forceinline__ bool sw_bond_active(const SwLaunch& P, const int8_t* s, uint32_t i, uint32_t j,
                                               uint32_t mu, uint32_t r, uint32_t c3) {
    const uint32_t b = P.dim * i + mu;
    if (s[i] != s[j]) return false;
    const uint4 w = philox4x32_10(make_uint4(b >> 2, P.t, r, c3), (uint32_t)P.seed, (uint32_t)(P.seed >> 32));
    const uint32_t u = (b & 3u) == 0 ? w.x : (b & 3u) == 1 ? w.y : (b & 3u) == 2 ? w.z : w.w;
    return (long long)u <= P.T_bond;
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

template <uint32_t DIM>
__global__ void __launch_bounds__(256) k_sw_bonds(const __grid_constant__ SwLaunch P) {
    const uint64_t copy = P.copy0 + blockIdx.y;
    const uint32_t i0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (i0 >= P.N) return;
    const int8_t* s = P.spins + copy * P.N;
    uint8_t* bonds = P.bonds + copy * P.N;
    uint32_t* par = P.parent + copy * P.N;
    uint32_t inst, r;
    split_copy(copy, P.R, inst, r);
    const uint32_t c3 = c3_word(kPurposeSwBond, 0u, P.inst_base + inst);
    uint32_t flags[4];
    sw_bond_flags<DIM>(P, s, i0, r, c3, flags);
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

template <uint32_t DIM>
__global__ void __launch_bounds__(256) k_sw_local(const __grid_constant__ SwLaunch P) {
    __shared__ uint32_t lp[1024];
    const uint64_t copy = P.copy0 + blockIdx.y;
    const int8_t* s = P.spins + copy * P.N;
    uint32_t inst, r;
    split_copy(copy, P.R, inst, r);
    const uint32_t c3 = c3_word(kPurposeSwBond, 0u, P.inst_base + inst);
    const SwTile T = sw_tile(DIM);
    const uint32_t ntx = P.L / T.tx, nty = P.L / T.ty;
    const uint32_t bx = blockIdx.x % ntx, by = (blockIdx.x / ntx) % nty, bz = blockIdx.x / (ntx * nty);
    // thread t: local sites l = 4t .. 4t+3 (consecutive x in one tile row)
    const uint32_t l0 = 4 * threadIdx.x;
    const uint32_t lx = l0 % T.tx, ly = (l0 / T.tx) % T.ty, lz = l0 / (T.tx * T.ty);
    const uint32_t i0 = ((bz * T.tz + lz) * P.L + by * T.ty + ly) * P.L + bx * T.tx + lx;
    uint32_t flags[4];
    sw_bond_flags_row<DIM>(P, s, i0, bx * T.tx + lx, by * T.ty + ly, bz * T.tz + lz, r, c3, flags);
    // runs along x: a site starts a run at x == 0 or where the bond from its
    // left neighbour is inactive. Each site's first parent is the start of its
    // run (a tile row spans TPR lanes of one warp: its run starts form one
    // 32-bit mask), so only the bonds along y (and z) go through the union-find.
    constexpr uint32_t TPR = (DIM == 2 ? 32u : 16u) / 4u;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t left = __shfl_up_sync(0xffffffffu, flags[3] & 1u, 1);  // bond into this thread's first site
    uint32_t starts = (lx == 0 || !left) ? 1u : 0u;
#pragma unroll
    for (int k = 1; k < 4; ++k) starts |= (flags[k - 1] & 1u) ? 0u : 1u << k;
    starts <<= 4 * (lane % TPR);
#pragma unroll
    for (uint32_t o = 1; o < TPR; o <<= 1) starts |= __shfl_xor_sync(0xffffffffu, starts, o);
#pragma unroll
    for (uint32_t k = 0; k < 4; ++k)  // bit 0 (x == 0) is always set
        lp[l0 + k] = l0 - lx + 31u - __clz(starts & ((2u << (lx + k)) - 1u));
    __syncthreads();
    // bonds along y and z inside the tile: unite in shared memory
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint32_t l = l0 + k;
        if ((flags[k] & 2u) && ly + 1 < T.ty) sw_unite<false>(lp, l, l + T.tx, P.err);
        if ((flags[k] & 4u) && lz + 1 < T.tz) sw_unite<false>(lp, l, l + T.tx * T.ty, P.err);
    }
    __syncthreads();
    uint32_t g[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint32_t root = sw_find<false>(lp, l0 + k);
        const uint32_t rx = root % T.tx, ry = (root / T.tx) % T.ty, rz = root / (T.tx * T.ty);
        g[k] = ((bz * T.tz + rz) * P.L + by * T.ty + ry) * P.L + bx * T.tx + rx;
    }
    // i0 % 4 == 0, N % 4 == 0 and the forest is a cudaMalloc block: 16-byte aligned
    *reinterpret_cast<uint4*>(P.parent + copy * P.N + i0) = make_uint4(g[0], g[1], g[2], g[3]);
}

// First site of the run holding site x (run-start mask R of the row; bit 0 is always set).
__device__ __forceinline__ uint32_t sw_run_start(uint32_t R, uint32_t x) {
    return 31u - __clz(R & (0xFFFFFFFFu >> (31u - x)));
}

// 2D tiles, the labelling by runs: as k_sw_local<2> (thread t: sites 4t .. 4t+3,
// eight lanes per tile row), with the union-find over run starts only. A row's
// run starts and y bonds become 32-bit masks; a y bond unites the runs holding
// its two ends, and one union per pair of overlapping runs suffices (the bond
// at x joins the same pair as the one at x - 1 unless a run starts at x in
// either row); the root of each run is found once, at its start, and every site
// takes its run's root.
// Appends the items with has = true of the warp's lanes to the warp's queue q
// (lane order), advancing n; all 32 lanes call it together.
__device__ __forceinline__ void sw_warp_push(uint32_t* q, uint32_t& n, bool has, uint32_t item) {
    const uint32_t b = __ballot_sync(0xffffffffu, has);
    if (has) q[n + __popc(b & ((1u << (threadIdx.x & 31u)) - 1u))] = item;
    n += __popc(b);
}

__global__ void __launch_bounds__(256) k_sw_local_runs(const __grid_constant__ SwLaunch P) {
    __shared__ uint32_t lp[1024];
    __shared__ uint16_t rt[1024];    // root of each run, at its start
    __shared__ uint32_t rmask[32];   // run starts of each tile row
    __shared__ uint32_t queue[8][128];  // per warp: unions (a | b << 16), then run starts
    const uint64_t copy = P.copy0 + blockIdx.y;
    const int8_t* s = P.spins + copy * P.N;
    uint32_t inst, r;
    split_copy(copy, P.R, inst, r);
    const uint32_t c3 = c3_word(kPurposeSwBond, 0u, P.inst_base + inst);
    const uint32_t L = P.L, ntx = L / 32u;
    const uint32_t bx = blockIdx.x % ntx, by = blockIdx.x / ntx;
    const uint32_t l0 = 4 * threadIdx.x, lx = l0 & 31u, ly = l0 >> 5, row = l0 - lx;
    const uint32_t i0 = (by * 32u + ly) * L + bx * 32u + lx;
    uint32_t flags[4];
    sw_bond_flags_row<2>(P, s, i0, bx * 32u + lx, by * 32u + ly, 0u, r, c3, flags);
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t left = __shfl_up_sync(0xffffffffu, flags[3] & 1u, 1);  // bond into this thread's first site
    uint32_t R = (lx == 0 || !left) ? 1u : 0u, Y = 0u;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (k > 0) R |= (flags[k - 1] & 1u) ? 0u : 1u << k;
        Y |= (flags[k] & 2u) ? 1u << k : 0u;
    }
    R <<= 4 * (lane & 7u);
    Y <<= 4 * (lane & 7u);
#pragma unroll
    for (uint32_t o = 1; o < 8u; o <<= 1) {
        R |= __shfl_xor_sync(0xffffffffu, R, o);
        Y |= __shfl_xor_sync(0xffffffffu, Y, o);
    }
    if ((lane & 7u) == 0) rmask[ly] = R;
#pragma unroll
    for (uint32_t k = 0; k < 4; ++k)
        if ((R >> (lx + k)) & 1u) lp[l0 + k] = l0 + k;  // run starts are their own parents
    __syncthreads();
    // the warp's unions, then its run starts, go through a queue so that every
    // lane works on one at a time (instead of each lane on its own few sites)
    uint32_t* q = queue[threadIdx.x >> 5];
    uint32_t n = 0;
    {
        const uint32_t Rn = ly < 31u ? rmask[ly + 1] : 0u;
        const uint32_t U = ly < 31u ? Y & ~((Y << 1) & ~R & ~Rn) : 0u;
#pragma unroll
        for (uint32_t k = 0; k < 4; ++k) {
            const uint32_t x = lx + k;
            const bool has = (U >> x) & 1u;
            sw_warp_push(q, n, has,
                         has ? (row + sw_run_start(R, x)) | ((row + 32u + sw_run_start(Rn, x)) << 16) : 0u);
        }
    }
    __syncwarp();
    for (uint32_t i = lane; i < n; i += 32u) sw_unite<false>(lp, q[i] & 0xFFFFu, q[i] >> 16, P.err);
    __syncthreads();
    n = 0;
#pragma unroll
    for (uint32_t k = 0; k < 4; ++k) sw_warp_push(q, n, (R >> (lx + k)) & 1u, l0 + k);
    __syncwarp();
    for (uint32_t i = lane; i < n; i += 32u) rt[q[i]] = (uint16_t)sw_find<false>(lp, q[i]);
    __syncthreads();
    uint32_t g[4];
#pragma unroll
    for (uint32_t k = 0; k < 4; ++k) {
        const uint32_t root = rt[row + sw_run_start(R, lx + k)];
        g[k] = (by * 32u + (root >> 5)) * L + bx * 32u + (root & 31u);
    }
    // i0 % 4 == 0, N % 4 == 0 and the forest is a cudaMalloc block: 16-byte aligned
    *reinterpret_cast<uint4*>(P.parent + copy * P.N + i0) = make_uint4(g[0], g[1], g[2], g[3]);
}

// The bonds that leave their tile: e < N / tx are the sites with x % tx == tx - 1
// (bond along x), then N / ty sites with y % ty == ty - 1 (along y), then in 3D
// N / tz sites with z % tz == tz - 1 (along z).
__host__ __device__ __forceinline__ uint32_t sw_cross_count(uint32_t N, uint32_t dim) {
    return dim == 2 ? N / 32 + N / 32 : N / 16 + N / 8 + N / 8;
}

__global__ void __launch_bounds__(256) k_sw_cross(const __grid_constant__ SwLaunch P) {
    const uint64_t copy = P.copy0 + blockIdx.y;
    uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= sw_cross_count(P.N, P.dim)) return;
    const SwTile T = sw_tile(P.dim);
    const uint32_t L = P.L, LL = L * L;
    uint32_t i, j, mu;
    if (e < P.N / T.tx) {  // (row, tile column) -> x = tx c + tx - 1
        const uint32_t nc = L / T.tx, row = e / nc, x = (e - row * nc) * T.tx + T.tx - 1;
        i = row * L + x;
        j = x + 1 == L ? i - x : i + 1;
        mu = 0;
    } else if ((e -= P.N / T.tx) < P.N / T.ty) {  // (z, tile row k, x) -> y = ty k + ty - 1
        const uint32_t nk = L / T.ty, rest = e / L, x = e - rest * L, z = rest / nk, y = (rest - z * nk) * T.ty + T.ty - 1;
        i = (z * L + y) * L + x;
        j = y + 1 == L ? i - (L - 1) * L : i + L;
        mu = 1;
    } else {  // (tile layer k, y, x) -> z = tz k + tz - 1
        e -= P.N / T.ty;
        const uint32_t k = e / LL, z = k * T.tz + T.tz - 1;
        i = z * LL + (e - k * LL);
        j = z + 1 == L ? i - (L - 1) * LL : i + LL;
        mu = 2;
    }
    const int8_t* s = P.spins + copy * P.N;
    uint32_t inst, r;
    split_copy(copy, P.R, inst, r);
    if (sw_bond_active(P, s, i, j, mu, r, c3_word(kPurposeSwBond, 0u, P.inst_base + inst)))
        sw_unite<true>(P.parent + copy * P.N, i, j, P.err);
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
    uint32_t inst, r;
    split_copy(copy, P.R, inst, r);
    const uint4 w = philox4x32_10(make_uint4(root >> 2, P.t, r, c3_word(kPurposeSwFlip, 0u, P.inst_base + inst)),
                                  (uint32_t)P.seed, (uint32_t)(P.seed >> 32));
    const uint32_t word = (root & 3u) == 0 ? w.x : (root & 3u) == 1 ? w.y : (root & 3u) == 2 ? w.z : w.w;
    if (word >> 31) P.spins[copy * P.N + i] = (int8_t)(-P.spins[copy * P.N + i]);
    if (P.labels) P.labels[copy * P.N + i] = (int32_t)root;
}

__device__ __forceinline__ uint32_t sw_coin(const PhiloxFixed& pf, uint32_t root) {
    const uint4 w = philox_q_wide(pf, root >> 2);
    const uint32_t word = (root & 3u) == 0 ? w.x : (root & 3u) == 1 ? w.y : (root & 3u) == 2 ? w.z : w.w;
    return word >> 31;
}

__global__ void __launch_bounds__(256) k_sw_flip_tiled(const __grid_constant__ SwLaunch P) {
    __shared__ uint32_t tpar[1024];   // the tile's parent pointers (global site indices)
    __shared__ uint32_t troot[1024];  // root of each end node
    __shared__ uint8_t tcoin[1024];   // its coin (1: the cluster flips)
    __shared__ uint32_t tqueue[8][128];  // per warp: its end nodes (local indices)
    const uint64_t copy = P.copy0 + blockIdx.y;
    uint32_t inst, r;
    split_copy(copy, P.R, inst, r);
    const SwTile T = sw_tile(P.dim);
    const uint32_t L = P.L, ntx = L / T.tx, nty = L / T.ty;
    const uint32_t bx = blockIdx.x % ntx, by = (blockIdx.x / ntx) % nty, bz = blockIdx.x / (ntx * nty);
    const uint32_t l0 = 4 * threadIdx.x;
    const uint32_t lx = l0 % T.tx, ly = (l0 / T.tx) % T.ty, lz = l0 / (T.tx * T.ty);
    const uint32_t i0 = ((bz * T.tz + lz) * L + by * T.ty + ly) * L + bx * T.tx + lx;
    uint32_t* par = P.parent + copy * P.N;
    const uint4 p4 = __ldcg(reinterpret_cast<const uint4*>(par + i0));
    tpar[l0] = p4.x;
    tpar[l0 + 1] = p4.y;
    tpar[l0 + 2] = p4.z;
    tpar[l0 + 3] = p4.w;
    __syncthreads();
    // each site's chain inside the tile (pointers strictly decrease until a
    // root, so at most 1024 steps) ends at node `end`: a root, or a node whose
    // parent lies in another tile
    uint32_t end[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        uint32_t cl = l0 + k, cg = i0 + k;
        for (uint32_t n = 0; n < 1024; ++n) {
            const uint32_t p = tpar[cl];
            if (p == cg) break;
            uint32_t px, py, pz;
            if (P.lshift) {  // L = 2^lshift
                px = p & (L - 1);
                py = (p >> P.lshift) & (L - 1);
                pz = p >> (2 * P.lshift);
            } else {
                const uint32_t row = p / L;
                px = p - row * L;
                py = row % L;
                pz = row / L;
            }
            if (px / T.tx != bx || py / T.ty != by || pz / T.tz != bz) break;
            cl = ((pz - bz * T.tz) * T.ty + (py - by * T.ty)) * T.tx + (px - bx * T.tx);
            cg = p;
        }
        end[k] = cl;
    }
    // end nodes: the root in the global forest and its coin, through a per-warp
    // queue so that every lane works on one end node at a time
    const PhiloxFixed pf = philox_fix(P.t, r, c3_word(kPurposeSwFlip, 0u, P.inst_base + inst), (uint32_t)P.seed,
                                      (uint32_t)(P.seed >> 32));
    uint32_t* q = tqueue[threadIdx.x >> 5];
    uint32_t n = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) sw_warp_push(q, n, end[k] == l0 + k, l0 + k);
    __syncwarp();
    for (uint32_t i = threadIdx.x & 31u; i < n; i += 32u) {
        const uint32_t l = q[i];
        const uint32_t ex = l % T.tx, ey = (l / T.tx) % T.ty, ez = l / (T.tx * T.ty);
        const uint32_t gl = ((bz * T.tz + ez) * L + by * T.ty + ey) * L + bx * T.tx + ex;  // its global index
        const uint32_t p = tpar[l];
        const uint32_t root = p == gl ? p : sw_find<true>(par, p);
        troot[l] = root;
        tcoin[l] = (uint8_t)sw_coin(pf, root);
    }
    __syncthreads();
    // i0 % 4 == 0 and the spin buffer is 16-byte aligned: one word per thread
    uint32_t* sw = reinterpret_cast<uint32_t*>(P.spins + copy * P.N + i0);
    uint32_t w = *sw;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (!tcoin[end[k]]) continue;
        const uint32_t b = (uint32_t)(uint8_t)(-(int8_t)(w >> (8 * k)));
        w = (w & ~(0xFFu << (8 * k))) | (b << (8 * k));
    }
    *sw = w;
    if (P.labels) {
#pragma unroll
        for (int k = 0; k < 4; ++k) P.labels[copy * P.N + i0 + k] = (int32_t)troot[end[k]];
    }
}

cudaError_t launch_sw_update(const SwLaunch& P0, uint64_t copies, cudaStream_t s) {
    if (P0.N % 4 != 0) return cudaErrorInvalidValue;
    for (uint64_t c0 = 0; c0 < copies; c0 += 65535) {
        SwLaunch P = P0;
        P.copy0 = c0;
        const uint32_t nc = (uint32_t)((copies - c0) < 65535 ? (copies - c0) : 65535);
        const uint32_t quads = P.N / 4;
        const bool tiled = sw_tiled(P.dim, P.L);
        cudaError_t e;
        if (tiled) {
            if (P.dim == 2) k_sw_local_runs<<<dim3(P.N / 1024, nc), 256, 0, s>>>(P);
            else k_sw_local<3><<<dim3(P.N / 1024, nc), 256, 0, s>>>(P);
            count_launch();
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            k_sw_cross<<<dim3((sw_cross_count(P.N, P.dim) + 255) / 256, nc), 256, 0, s>>>(P);
            count_launch();
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            k_sw_flip_tiled<<<dim3(P.N / 1024, nc), 256, 0, s>>>(P);
            count_launch();
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            continue;
        } else {
            if (P.dim == 2) k_sw_bonds<2><<<dim3((quads + 255) / 256, nc), 256, 0, s>>>(P);
            else k_sw_bonds<3><<<dim3((quads + 255) / 256, nc), 256, 0, s>>>(P);
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
