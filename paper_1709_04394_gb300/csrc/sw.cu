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
// Tiled labelling of 3D lattices (L % 16 == 0: 16 x 8 x 8 tiles), the tile
// decomposition of Sec. 3.3 with the consolidation done by atomics:
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
//
// 2D lattices with L % 32 == 0 take 32 x 32 tiles with a scanline labelling,
// the tile labels kept apart from the global forest:
//  k_sw_scan2    : one warp per tile, lane x = column x, the rows in order.
//                  Row r's x bonds cut it into runs; a run's label is the
//                  smallest of its start and of the labels its y bonds reach in
//                  row r - 1, and a run that reaches two components above hooks
//                  the larger label under the smaller in the tile's label
//                  forest (shared memory). At the end every site's label is
//                  resolved to its component's smallest site: lab[i] = that
//                  site's tile-local index, and parent[g] = g for each such
//                  tile root g, the only nodes of the global forest;
//  k_sw_cross    : unites the tile roots of the two ends of each active
//                  tile-crossing bond in the global forest;
//  k_sw_flip_lab : one CTA per tile finds the global root of each tile root
//                  whose component touches the tile border (the others are
//                  roots of whole clusters) and draws each tile root's coin
//                  once; every site takes its tile root's.
#include "bits.cuh"
#include "check.cuh"
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

// Appends the items with has = true of the warp's lanes to the warp's queue q
// (lane order), advancing n; all 32 lanes call it together.
__device__ __forceinline__ void sw_warp_push(uint32_t* q, uint32_t& n, bool has, uint32_t item) {
    const uint32_t b = __ballot_sync(0xffffffffu, has);
    if (has) q[n + __popc(b & ((1u << (threadIdx.x & 31u)) - 1u))] = item;
    n += __popc(b);
}

// ---- 2D scanline tiles ----

constexpr uint32_t kSwScanWarps = 4;  // tiles (warps) per block of k_sw_scan2

// Global index of the 32 x 32 tile-local site k (k = 32 row + column) of the
// tile holding site i.
__device__ __forceinline__ uint32_t sw_tile_root(uint32_t k, uint32_t i, uint32_t L) {
    const uint32_t y = i / L, x = i - y * L;
    return ((y & ~31u) + (k >> 5)) * L + (x & ~31u) + (k & 31u);
}

__global__ void __launch_bounds__(32 * kSwScanWarps) k_sw_scan2(const __grid_constant__ SwLaunch P) {
    __shared__ uint32_t eq[kSwScanWarps][1024];       // label forest of each warp's tile (local indices)
    __shared__ uint16_t rowlab[kSwScanWarps][1024];   // each site's run label, resolved at the end
    const uint32_t lane = threadIdx.x & 31u, wib = threadIdx.x >> 5;
    const uint32_t L = P.L, ntx = L >> 5;
    const uint32_t tile = blockIdx.x * kSwScanWarps + wib;
    if (tile >= ntx * ntx) return;  // whole warp; no block barriers follow
    const uint64_t copy = P.copy0 + blockIdx.y;
    const int8_t* s = P.spins + copy * P.N;
    uint32_t inst, r;
    split_copy(copy, P.R, inst, r);
    const uint32_t bx = tile % ntx, by = tile / ntx, X = bx * 32u + lane;
    uint32_t* f = eq[wib];
    uint16_t* rl = rowlab[wib];
    // bond words: the forward bonds b = 2 i + mu of sites i = 2 q, 2 q + 1 are
    // the four words of Philox call q (t, replica and c3 hoisted)
    const PhiloxFixed pf = philox_fix(P.t, r, c3_word(kPurposeSwBond, 0u, P.inst_base + inst), (uint32_t)P.seed,
                                      (uint32_t)(P.seed >> 32));
    const long long Tb = P.T_bond;
    uint4 c = make_uint4(0u, 0u, 0u, 0u);
    int s_prev = 0;
    uint32_t w1_prev = 0u, lab_prev = 0u;
    for (uint32_t rr = 0; rr < 32u; ++rr) {
        const uint32_t y = by * 32u + rr;
        if ((rr & 1u) == 0u)  // lane l: the call of sites 2 (l & 15), +1 of row rr + l / 16
            c = philox_q_wide(pf, ((y + (lane >> 4)) * L + bx * 32u + 2u * (lane & 15u)) >> 1);
        const uint32_t src = ((rr & 1u) << 4) | (lane >> 1);
        const uint32_t a0 = __shfl_sync(0xffffffffu, c.x, src), a1 = __shfl_sync(0xffffffffu, c.y, src);
        const uint32_t a2 = __shfl_sync(0xffffffffu, c.z, src), a3 = __shfl_sync(0xffffffffu, c.w, src);
        const uint32_t w0 = (lane & 1u) ? a2 : a0;  // bond along x: word (2 i) & 3
        const uint32_t w1 = (lane & 1u) ? a3 : a1;  // bond along y: word (2 i + 1) & 3
        const int sc = s[GBMC_IDX((uint64_t)y * L + X, P.N)];
        const int sr = __shfl_down_sync(0xffffffffu, sc, 1);
        // the bond from lane 31 leaves the tile (k_sw_cross); so does the one into row 0
        const bool xb = lane < 31u && sc == sr && (long long)w0 <= Tb;
        const bool yb = rr > 0u && sc == s_prev && (long long)w1_prev <= Tb;
        const uint32_t R = ~(__ballot_sync(0xffffffffu, xb) << 1);  // run starts
        const uint32_t own = rr * 32u + lane;
        f[own] = own;
        const uint32_t la = yb ? sw_find<false>(f, lab_prev) : 0u;  // the component above, if reached
        // the run's label: segmented minimum over the run (lane x - d is in x's
        // run when no run starts at x - d + 1 .. x), then read at the run's end
        uint32_t v = yb ? la : own;
#pragma unroll
        for (uint32_t d = 1; d < 32u; d <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, v, d);
            if (lane >= d && ((R >> (lane - d + 1u)) & ((1u << d) - 1u)) == 0u) v = t < v ? t : v;
        }
        const uint32_t nxt = R & ~((2u << lane) - 1u);  // run starts right of this lane
        const uint32_t m = __shfl_sync(0xffffffffu, v, nxt ? (uint32_t)__ffs(nxt) - 2u : 31u);
        if (yb && la != m) sw_unite<false>(f, la, m, P.err);  // a second component above joins the run
        rl[own] = (uint16_t)m;
        lab_prev = m;
        s_prev = sc;
        w1_prev = w1;
        __syncwarp();
    }
    // every site's label resolved to its component's smallest site: lab = its
    // tile-local index; each tile root a node of the global forest
    uint32_t* par = P.parent + copy * P.N;
    uint16_t* lab = P.lab + copy * P.N;
    for (uint32_t rr = 0; rr < 32u; ++rr) {
        const uint32_t own = rr * 32u + lane, i = (by * 32u + rr) * L + X;
        const uint32_t root = sw_find<false>(f, rl[own]);
        lab[GBMC_IDX(i, P.N)] = (uint16_t)root;
        if (root == own) par[GBMC_IDX(i, P.N)] = i;
    }
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
    if (!sw_bond_active(P, s, i, j, mu, r, c3_word(kPurposeSwBond, 0u, P.inst_base + inst))) return;
    if (P.lab) {  // 2D scanline tiles: the ends' tile roots
        const uint16_t* lab = P.lab + copy * P.N;
        i = sw_tile_root(lab[i], i, L);
        j = sw_tile_root(lab[j], j, L);
    }
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

__global__ void __launch_bounds__(256) k_sw_flip_lab(const __grid_constant__ SwLaunch P) {
    __shared__ uint32_t troot[1024];     // global root of each tile root (by local index)
    __shared__ uint8_t tcoin[1024];      // its coin (1: the cluster flips)
    __shared__ uint32_t tqueue[8][128];  // per warp: its tile roots (local indices)
    __shared__ uint32_t tedge[32];       // the tile roots whose component touches the tile border
    const uint64_t copy = P.copy0 + blockIdx.y;
    uint32_t inst, r;
    split_copy(copy, P.R, inst, r);
    const uint32_t L = P.L, ntx = L >> 5;
    const uint32_t bx = blockIdx.x % ntx, by = blockIdx.x / ntx;
    const uint32_t l0 = 4 * threadIdx.x, lx = l0 & 31u, ly = l0 >> 5;
    const uint32_t i0 = (by * 32u + ly) * L + bx * 32u + lx;
    // i0 % 4 == 0 and the label buffer is a cudaMalloc block: 8-byte aligned
    const uint2 lv = *reinterpret_cast<const uint2*>(P.lab + copy * P.N + GBMC_IDX(i0, P.N));
    // i0 % 4 == 0 and the spin buffer is 16-byte aligned: one word per thread, loaded early
    uint32_t* sw = reinterpret_cast<uint32_t*>(P.spins + copy * P.N + i0);
    uint32_t w = *sw;
    const uint32_t k[4] = {lv.x & 0xFFFFu, lv.x >> 16, lv.y & 0xFFFFu, lv.y >> 16};
    // the tile roots whose component has a site on the tile border: only
    // they can have been united with other tiles' components
    if (threadIdx.x < 32u) tedge[threadIdx.x] = 0u;
    __syncthreads();
#pragma unroll
    for (uint32_t j = 0; j < 4; ++j)
        if (ly == 0u || ly == 31u || lx + j == 0u || lx + j == 31u) atomicOr(&tedge[k[j] >> 5], 1u << (k[j] & 31u));
    __syncthreads();
    // the tile roots: their global root and coin, through a per-warp queue so
    // that every lane works on one at a time
    const PhiloxFixed pf = philox_fix(P.t, r, c3_word(kPurposeSwFlip, 0u, P.inst_base + inst), (uint32_t)P.seed,
                                      (uint32_t)(P.seed >> 32));
    uint32_t* par = P.parent + copy * P.N;
    uint32_t* q = tqueue[threadIdx.x >> 5];
    uint32_t n = 0;
#pragma unroll
    for (uint32_t j = 0; j < 4; ++j) sw_warp_push(q, n, k[j] == l0 + j, l0 + j);
    __syncwarp();
    for (uint32_t a = threadIdx.x & 31u; a < n; a += 32u) {
        const uint32_t l = q[a];
        const uint32_t g = (by * 32u + (l >> 5)) * L + bx * 32u + (l & 31u);
        // a component away from the tile border is a whole cluster, rooted at g
        const uint32_t root = ((tedge[l >> 5] >> (l & 31u)) & 1u) ? sw_find<true>(par, g) : g;
        troot[l] = root;
        tcoin[l] = (uint8_t)sw_coin(pf, root);
    }
    __syncthreads();
#pragma unroll
    for (uint32_t j = 0; j < 4; ++j) {
        if (!tcoin[GBMC_IDX(k[j], 1024u)]) continue;
        const uint32_t b = (uint32_t)(uint8_t)(-(int8_t)(w >> (8 * j)));
        w = (w & ~(0xFFu << (8 * j))) | (b << (8 * j));
    }
    *sw = w;
    if (P.labels) {
#pragma unroll
        for (uint32_t j = 0; j < 4; ++j) P.labels[copy * P.N + i0 + j] = (int32_t)troot[GBMC_IDX(k[j], 1024u)];
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
        if (tiled && P.dim == 2) {
            if (!P.lab) return cudaErrorInvalidValue;
            const uint32_t tiles = P.N / 1024;
            k_sw_scan2<<<dim3((tiles + kSwScanWarps - 1) / kSwScanWarps, nc), 32 * kSwScanWarps, 0, s>>>(P);
            count_launch();
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            k_sw_cross<<<dim3((sw_cross_count(P.N, P.dim) + 255) / 256, nc), 256, 0, s>>>(P);
            count_launch();
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            k_sw_flip_lab<<<dim3(tiles, nc), 256, 0, s>>>(P);
            count_launch();
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            continue;
        }
        P.lab = nullptr;
        if (tiled) {
            k_sw_local<3><<<dim3(P.N / 1024, nc), 256, 0, s>>>(P);
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
