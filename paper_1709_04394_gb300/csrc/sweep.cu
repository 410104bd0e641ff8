// sweep.cu -- checkerboard Metropolis sweeps (Sec. 3.1, Eq. (8)) of int8
// lattices with per-site Philox words, for the ferromagnet (Eq. (7), J = 1)
// and the bimodal +-J spin glass (Sec. 6).
//
// Two kernels:
//  * k_sweep_resident: every copy of the lattice fits in one CTA's shared
//    memory. The CTA loads its copies (through the resampling gather of Sec.
//    5.4 when a parent map is given), runs all requested sweeps (colour 0,
//    then colour 1, with a CTA barrier between the half-sweeps) on the shared
//    copy, and writes them back once. Energy and magnetisation are taken in the
//    colour-1 pass of a measured sweep: every bond has exactly one odd end, so
//    E = -sum_{i odd} s_i h_i after the update, and every even site is the right
//    neighbour of exactly one odd site.
//  * k_halfsweep_global: one colour of one sweep straight on global memory, for
//    lattices too large for shared memory (one launch per half-sweep, the
//    kernel-boundary synchronisation described in Sec. 3.1).
//
// Spins are bytes +1 (0x01) / -1 (0xFF). For L % 8 == 0 the resident kernel
// keeps each copy in shared memory as two colour planes (the separate
// sub-lattice storage of Sec. 3.1): plane c, row r = z*L + y, holds the L/2
// sites of colour c of that row in x order. A thread updates one 32-bit word
// of a plane = 4 consecutive same-colour sites = the 4 words of one Philox
// call. Their vertical neighbours are the same word of the other plane in the
// rows above/below; the horizontal ones are the same word and the word shifted
// by one byte (funnel shift). Byte-parallel (s_i ^ s_j) & 4 summed over the
// neighbours gives 4a per site, a = number of unsatisfied bonds
// (s_i J_ij s_j = -1), so dE = 4 (dim - a); 4a is also the byte offset of the
// site's threshold in a shared table (dE <= 0 -> 0xffffffff, i.e. always
// accept), and the site flips iff u <= table[a]. The global-memory kernel
// works on the row-major layout with 8-byte chunks; L % 8 != 0 uses a per-site
// path with the same Philox words.
#include "device.cuh"
#include "internal.h"

namespace gbmc {

__device__ __forceinline__ uint64_t down_bits(uint64_t w) { return (w >> 1) & 0x0101010101010101ull; }

template <typename P>
__device__ __forceinline__ uint64_t ld8(const P* p) {
    return *reinterpret_cast<const uint64_t*>(p);
}

struct Thr {
    uint32_t t4, t8, t12;
};

// One 8-site chunk (row `row`, chunk `g`) of one copy: update the 4 sites of
// `colour`. sp: copy base; jb: bond planes of its instance (or null).
template <int DIM, bool EA, bool MEASURE>
__device__ __forceinline__ void unit_swar(uint8_t* sp, const uint8_t* jb, uint32_t L, uint32_t N,
                                          uint32_t row, uint32_t g, uint32_t colour,
                                          const PhiloxFixed& pf, const Thr& T, bool flip, int& e_acc,
                                          int& m_acc) {
    const uint32_t G = L >> 3;
    const uint32_t y = DIM == 3 ? row % L : row;
    const uint32_t z = DIM == 3 ? row / L : 0;
    const uint32_t off = (y + z + colour) & 1u;
    const uint32_t base = row * L;
    const uint32_t gl = g == 0 ? G - 1 : g - 1;
    const uint32_t gr = g + 1 == G ? 0 : g + 1;
    const uint32_t rowu = y == 0 ? row + L - 1 : row - 1;       // y - 1
    const uint32_t rowd = y + 1 == L ? row + 1 - L : row + 1;   // y + 1
    const uint64_t cur = ld8(sp + base + 8 * g);
    const uint64_t prv = ld8(sp + base + 8 * gl);
    const uint64_t nxt = ld8(sp + base + 8 * gr);
    const uint64_t up = ld8(sp + rowu * L + 8 * g);
    const uint64_t dn = ld8(sp + rowd * L + 8 * g);
    const uint64_t dc = down_bits(cur);
    uint64_t lft = down_bits((cur << 8) | (prv >> 56));
    uint64_t rgt = down_bits((cur >> 8) | (nxt << 56));
    uint64_t upb = down_bits(up), dnb = down_bits(dn);
    uint64_t bkb = 0, frb = 0;
    uint32_t rowb = 0;
    if (DIM == 3) {
        rowb = z == 0 ? row + (L - 1) * L : row - L;              // z - 1
        const uint32_t rowf = z + 1 == L ? row - (L - 1) * L : row + L;  // z + 1
        bkb = down_bits(ld8(sp + rowb * L + 8 * g));
        frb = down_bits(ld8(sp + rowf * L + 8 * g));
    }
    if (EA) {
        // bond planes: byte 1 where J = -1; an unsatisfied bond has d_i ^ d_j ^ b = 1
        const uint64_t jx = ld8(jb + base + 8 * g);
        const uint64_t jxp = ld8(jb + base + 8 * gl);
        rgt ^= jx;
        lft ^= (jx << 8) | (jxp >> 56);
        dnb ^= ld8(jb + N + base + 8 * g);
        upb ^= ld8(jb + N + rowu * L + 8 * g);
        if (DIM == 3) {
            frb ^= ld8(jb + 2 * N + base + 8 * g);
            bkb ^= ld8(jb + 2 * N + rowb * L + 8 * g);
        }
    }
    uint64_t a = (dc ^ lft) + (dc ^ rgt) + (dc ^ upb) + (dc ^ dnb);
    if (DIM == 3) a += (dc ^ bkb) + (dc ^ frb);

    uint4 w = make_uint4(0, 0, 0, 0);
    if (flip) w = philox_q(pf, row * G + g);
    uint64_t mask = 0;
    int e = 0;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const uint32_t pos = off + 2 * m;
        const int am = (int)((a >> (8 * pos)) & 0xFFu);
        const int d = DIM - am;  // dE / 4
        const uint32_t u = m == 0 ? w.x : m == 1 ? w.y : m == 2 ? w.z : w.w;
        const uint32_t thr = d == 1 ? T.t4 : (d == 2 ? T.t8 : T.t12);
        const bool acc = flip && (d <= 0 || u <= thr);
        mask |= acc ? (0xFEull << (8 * pos)) : 0ull;
        if (MEASURE) {
            const int sh = 2 * DIM - 2 * am;  // s_i h_i before the update
            e += acc ? sh : -sh;
        }
    }
    const uint64_t nw = cur ^ mask;
    if (flip) *reinterpret_cast<uint64_t*>(sp + base + 8 * g) = nw;
    if (MEASURE) {
        e_acc += e;
        m_acc += 8 - 2 * (int)__popcll(down_bits(nw));
    }
}

__device__ __forceinline__ uint32_t neq4(uint32_t a, uint32_t b) { return (a ^ b) & 0x04040404u; }

// Split-plane unit: word g of row `row` of colour plane `colour`; q is the
// Philox counter word of its 4 sites (row-major rank of the word over the
// whole lattice, which differs from row * (L/8) + g inside a tile). sp: copy
// base (plane 0 then plane 1, N/2 bytes each); jb: this colour's 2*DIM bond
// planes (bytes 0x04 where J = -1; order same-j x, shifted x, y-1, y+1, z-1,
// z+1); tbl: byte-addressed threshold table (entry a at byte 4a).
template <int DIM, bool EA, bool MEASURE>
__device__ __forceinline__ void unit_split(uint8_t* sp, const uint8_t* jb, uint32_t L, uint32_t N,
                                           uint32_t row, uint32_t y, uint32_t z, uint32_t g, uint32_t colour,
                                           const PhiloxFixed& pf, const uint8_t* tbl, bool doflip, int& e_acc,
                                           int& m_acc, uint32_t q) {
    const uint32_t W = L >> 3, H = N >> 1;
    const uint32_t o = (y + z + colour) & 1u;
    uint32_t* own = reinterpret_cast<uint32_t*>(sp + colour * H);
    const uint32_t* oth = reinterpret_cast<const uint32_t*>(sp + (colour ^ 1u) * H);
    const uint32_t rw = row * W;
    const uint32_t cur = own[rw + g];
    const uint32_t same = oth[rw + g];
    // horizontal neighbour not sharing j: j+1 (odd x) or j-1 (even x)
    const uint32_t side = o ? __funnelshift_r(same, oth[rw + (g + 1 == W ? 0 : g + 1)], 8)
                            : __funnelshift_l(oth[rw + (g == 0 ? W - 1 : g - 1)], same, 8);
    const uint32_t rowu = y == 0 ? row + L - 1 : row - 1;
    const uint32_t rowd = y + 1 == L ? row + 1 - L : row + 1;
    const uint32_t up = oth[rowu * W + g], dn = oth[rowd * W + g];
    uint32_t a4;
    const uint32_t* b = EA ? reinterpret_cast<const uint32_t*>(jb) + rw + g : nullptr;
    const uint32_t P = H >> 2;  // words per plane
    if (EA) {
        a4 = (neq4(cur, same) ^ b[0]) + (neq4(cur, side) ^ b[P]) + (neq4(cur, up) ^ b[2 * P]) +
             (neq4(cur, dn) ^ b[3 * P]);
    } else {
        a4 = neq4(cur, same) + neq4(cur, side) + neq4(cur, up) + neq4(cur, dn);
    }
    if (DIM == 3) {
        const uint32_t rowb = z == 0 ? row + (L - 1) * L : row - L;
        const uint32_t rowf = z + 1 == L ? row - (L - 1) * L : row + L;
        const uint32_t bk = oth[rowb * W + g], fr = oth[rowf * W + g];
        if (EA) a4 += (neq4(cur, bk) ^ b[4 * P]) + (neq4(cur, fr) ^ b[5 * P]);
        else a4 += neq4(cur, bk) + neq4(cur, fr);
    }
    uint32_t flip = 0;
    if (doflip) {
        const uint4 w = philox_q(pf, q);
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const uint32_t am = __byte_perm(a4, 0u, 0x4440u + m);  // 4a of site m
            const uint32_t thr = *reinterpret_cast<const uint32_t*>(tbl + am);
            const uint32_t u = m == 0 ? w.x : m == 1 ? w.y : m == 2 ? w.z : w.w;
            flip |= (u <= thr) ? (0xFEu << (8 * m)) : 0u;
        }
    }
    const uint32_t nw = cur ^ flip;
    if (doflip) own[rw + g] = nw;
    if (MEASURE) {
        // E contribution -sum s_new h = sum_acc s h - sum_rej s h, s h = 2 DIM - (4a)/2
        const int s_all = (int)__dp4a(a4, 0x01010101u, 0u);
        const int s_acc = (int)__dp4a(a4 & flip, 0x01010101u, 0u);
        const int nacc = __popc(flip & 0x02020202u);
        e_acc += 4 * DIM * nacc - s_acc - 8 * DIM + s_all / 2;
        // the other plane's word `same` pairs each of its sites with one site here
        m_acc += 8 - 2 * (__popc(nw & 0x02020202u) + __popc(same & 0x02020202u));
    }
}

// Per-site path for any even L: quad q covers colour ranks k = 4q .. 4q+3.
template <int DIM, bool EA, bool MEASURE>
__device__ __forceinline__ void unit_scalar(int8_t* sp, const uint8_t* jb, uint32_t L, uint32_t N,
                                            uint32_t q, uint32_t colour, const PhiloxFixed& pf,
                                            const Thr& T, bool flip, int& e_acc, int& m_acc) {
    const uint32_t half = L >> 1;
    const uint32_t ncol = N >> 1;
    uint4 w = make_uint4(0, 0, 0, 0);
    if (flip) w = philox_q(pf, q);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const uint32_t k = 4 * q + m;
        if (k >= ncol) break;
        const uint32_t row = k / half, j = k - row * half;
        const uint32_t y = DIM == 3 ? row % L : row;
        const uint32_t z = DIM == 3 ? row / L : 0;
        const uint32_t x = 2 * j + ((y + z + colour) & 1u);
        const uint32_t i = row * L + x;
        const uint32_t xl = x == 0 ? L - 1 : x - 1, xr = x + 1 == L ? 0 : x + 1;
        const uint32_t yu = y == 0 ? L - 1 : y - 1, yd = y + 1 == L ? 0 : y + 1;
        const uint32_t zb = DIM == 3 ? row - y : 0;  // z*L
        const uint32_t i_l = row * L + xl, i_r = row * L + xr;
        const uint32_t i_u = (zb + yu) * L + x, i_d = (zb + yd) * L + x;
        int jl = 1, jr = 1, ju = 1, jd = 1, jbk = 1, jf = 1;
        if (EA) {
            jr = jb[i] ? -1 : 1;
            jl = jb[i_l] ? -1 : 1;
            jd = jb[N + i] ? -1 : 1;
            ju = jb[N + i_u] ? -1 : 1;
        }
        int h = jl * sp[i_l] + jr * sp[i_r] + ju * sp[i_u] + jd * sp[i_d];
        if (DIM == 3) {
            const uint32_t zbk = z == 0 ? L - 1 : z - 1, zf = z + 1 == L ? 0 : z + 1;
            const uint32_t i_b = (zbk * L + y) * L + x, i_f = (zf * L + y) * L + x;
            if (EA) {
                jf = jb[2 * N + i] ? -1 : 1;
                jbk = jb[2 * N + i_b] ? -1 : 1;
            }
            h += jbk * sp[i_b] + jf * sp[i_f];
        }
        const int si = sp[i];
        const int dE = 2 * si * h;
        const uint32_t u = m == 0 ? w.x : m == 1 ? w.y : m == 2 ? w.z : w.w;
        const uint32_t thr = dE == 4 ? T.t4 : (dE == 8 ? T.t8 : T.t12);
        const bool acc = flip && (dE <= 0 || u <= thr);
        const int snew = acc ? -si : si;
        if (flip) sp[i] = (int8_t)snew;
        if (MEASURE) {
            e_acc -= snew * h;
            m_acc += snew + sp[i_r];
        }
    }
}

// Walk of one thread over the split-plane units of a copy: when the threads
// serving a copy are a multiple of the words per plane row, each thread keeps
// one word column g and steps through rows (no division in the loop).
struct UnitWalk {
    bool rowwise;
    uint32_t g0, row0, y0, z0, rstep, dy, dz;
};

template <int DIM>
__device__ __forceinline__ UnitWalk make_walk(uint32_t L, uint32_t lane, uint32_t tpr) {
    UnitWalk w;
    const uint32_t W = L >> 3;
    w.rowwise = (tpr % W) == 0;
    w.g0 = lane % W;
    w.row0 = lane / W;
    w.rstep = tpr / W;
    w.y0 = DIM == 3 ? w.row0 % L : w.row0;
    w.z0 = DIM == 3 ? w.row0 / L : 0;
    w.dy = DIM == 3 ? w.rstep % L : w.rstep;
    w.dz = DIM == 3 ? w.rstep / L : 0;
    return w;
}

template <int DIM, bool EA, bool SWAR, bool ROWWISE, bool MEASURE>
__device__ __forceinline__ void half_sweep_copy_m(uint8_t* sp, const uint8_t* jb, uint32_t L, uint32_t N,
                                                  uint32_t first_unit, uint32_t stride, const UnitWalk& wk,
                                                  uint32_t colour, const PhiloxFixed& pf, const Thr& T,
                                                  const uint8_t* tbl, bool flip, int& e, int& m) {
    if (SWAR) {
        const uint32_t W = L >> 3, rows = N / L;
        const uint8_t* jbc = EA ? jb + colour * (2u * DIM) * (N >> 1) : nullptr;
        if (ROWWISE) {
            uint32_t y = wk.y0, z = wk.z0;
#pragma unroll 4
            for (uint32_t row = wk.row0; row < rows; row += wk.rstep) {
                unit_split<DIM, EA, MEASURE>(sp, jbc, L, N, row, y, z, wk.g0, colour, pf, tbl, flip, e, m,
                                             row * W + wk.g0);
                if (DIM == 3) {
                    y += wk.dy;
                    z += wk.dz;
                    if (y >= L) {
                        y -= L;
                        ++z;
                    }
                } else {
                    y += wk.rstep;
                }
            }
        } else {
            const uint32_t units = N >> 3;
            for (uint32_t uu = first_unit; uu < units; uu += stride) {
                const uint32_t row = uu / W;
                unit_split<DIM, EA, MEASURE>(sp, jbc, L, N, row, DIM == 3 ? row % L : row, DIM == 3 ? row / L : 0,
                                             uu % W, colour, pf, tbl, flip, e, m, uu);
            }
        }
    } else {
        const uint32_t units = ((N >> 1) + 3) >> 2;
        int8_t* s8 = reinterpret_cast<int8_t*>(sp);
        for (uint32_t uu = first_unit; uu < units; uu += stride)
            unit_scalar<DIM, EA, MEASURE>(s8, jb, L, N, uu, colour, pf, T, flip, e, m);
    }
}

template <int DIM, bool EA, bool SWAR, bool ROWWISE>
__device__ __forceinline__ void half_sweep_copy(uint8_t* sp, const uint8_t* jb, uint32_t L, uint32_t N,
                                                uint32_t first_unit, uint32_t stride, const UnitWalk& wk,
                                                uint32_t colour, const PhiloxFixed& pf, const Thr& T,
                                                const uint8_t* tbl, bool flip, bool measure, int& e, int& m) {
    if (measure)
        half_sweep_copy_m<DIM, EA, SWAR, ROWWISE, true>(sp, jb, L, N, first_unit, stride, wk, colour, pf, T, tbl,
                                                        flip, e, m);
    else
        half_sweep_copy_m<DIM, EA, SWAR, ROWWISE, false>(sp, jb, L, N, first_unit, stride, wk, colour, pf, T, tbl,
                                                         flip, e, m);
}

__device__ __forceinline__ uint32_t padded(uint32_t n) { return (n + 15u) & ~15u; }

// Grid: one CTA per (job, instance, group of rpc replicas). blockDim.x must be
// a multiple of rpc; blockDim.x / rpc threads serve each replica. Shared
// memory: rpc copies (split colour planes when SWAR, else row-major), then
// the instance's bond planes (EA).
template <int DIM, bool EA, bool SWAR, bool ROWWISE>
__global__ void __launch_bounds__(256) k_sweep_resident(const __grid_constant__ SweepLaunch P) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ int acc_e[64], acc_m[64];
    __shared__ __align__(16) uint32_t s_tbl[8];
    __shared__ __align__(16) uint32_t s_tblc[64][8];  // per-copy tables (parallel tempering)
    int jid = 0;
    while (jid + 1 < P.njobs && blockIdx.x >= P.cta_begin[jid + 1]) ++jid;
    const SweepJob& J = P.jobs[jid];
    const uint32_t local = blockIdx.x - P.cta_begin[jid];
    const uint32_t inst = local / J.ctas_per_inst;
    const uint32_t r0 = (local - inst * J.ctas_per_inst) * J.rpc;
    const uint32_t nrep = min(J.rpc, J.R - r0);
    const uint32_t N = J.N, L = J.L, stride_b = padded(N);
    const uint64_t slot0 = (uint64_t)inst * J.R + r0;
    uint8_t* jsm = smem + (uint64_t)J.rpc * stride_b;

    // ---- load: copy c of this CTA from src + parent(c) (the resampling gather) ----
    if (SWAR) {
        // row-major global -> colour planes: the even-x bytes of row r belong
        // to colour (y+z)&1, the odd-x bytes to the other colour
        const uint32_t chunks = N >> 3, W = L >> 3, H = N >> 1;
        for (uint32_t idx = threadIdx.x; idx < nrep * chunks; idx += blockDim.x) {
            const uint32_t c = idx / chunks, ch = idx - c * chunks;
            const uint32_t row = ch / W;
            const uint64_t slot = slot0 + c;
            const uint64_t srcslot = J.parent ? (uint64_t)inst * J.R + J.parent[slot] : slot;
            const uint2 v = *reinterpret_cast<const uint2*>(J.src + srcslot * N + (uint64_t)ch * 8);
            const uint32_t y = DIM == 3 ? row % L : row, z = DIM == 3 ? row / L : 0;
            const uint32_t pe = (y + z) & 1u;
            uint32_t* pl = reinterpret_cast<uint32_t*>(smem + c * stride_b);
            pl[pe * (H >> 2) + ch] = __byte_perm(v.x, v.y, 0x6420);
            pl[(pe ^ 1u) * (H >> 2) + ch] = __byte_perm(v.x, v.y, 0x7531);
        }
        if (EA) {
            const uint4* jsrc = reinterpret_cast<const uint4*>(J.jsplit + (uint64_t)inst * 6 * N);
            for (uint32_t idx = threadIdx.x; idx < (6 * N) >> 4; idx += blockDim.x)
                reinterpret_cast<uint4*>(jsm)[idx] = jsrc[idx];
        }
    } else {
        const uint32_t nw = N >> 2;
        for (uint32_t idx = threadIdx.x; idx < nrep * nw; idx += blockDim.x) {
            const uint32_t c = idx / nw, wi = idx - c * nw;
            const uint64_t slot = slot0 + c;
            const uint64_t srcslot = J.parent ? (uint64_t)inst * J.R + J.parent[slot] : slot;
            reinterpret_cast<uint32_t*>(smem + c * stride_b)[wi] =
                reinterpret_cast<const uint32_t*>(J.src + srcslot * N)[wi];
        }
        if (EA) {
            const uint8_t* jsrc = J.jbits + (uint64_t)inst * 3 * N;
            const uint32_t nwj = (3 * N) >> 2;
            for (uint32_t idx = threadIdx.x; idx < nwj; idx += blockDim.x)
                reinterpret_cast<uint32_t*>(jsm)[idx] = reinterpret_cast<const uint32_t*>(jsrc)[idx];
        }
    }
    if (threadIdx.x < 64) {
        acc_e[threadIdx.x] = 0;
        acc_m[threadIdx.x] = 0;
    }
    if (threadIdx.x < 8) {
        // entry a (byte 4a): dE = 4 (DIM - a); dE <= 0 is always accepted
        const int d = DIM - (int)threadIdx.x;
        s_tbl[threadIdx.x] = d <= 0 ? 0xFFFFFFFFu : (d == 1 ? J.thr[0] : (d == 2 ? J.thr[1] : J.thr[2]));
    }
    if (J.temp_of) {
        // each copy at its own temperature: its own table
        for (uint32_t i = threadIdx.x; i < nrep * 8; i += blockDim.x) {
            const uint32_t c = i >> 3, a = i & 7u;
            const uint32_t* th = J.thr_temp + 3ull * J.temp_of[slot0 + c];
            const int d = DIM - (int)a;
            s_tblc[c][a] = d <= 0 ? 0xFFFFFFFFu : th[d - 1];
        }
    }
    __syncthreads();

    const uint32_t tpr = blockDim.x / J.rpc;
    const uint32_t c = threadIdx.x / tpr;  // copy served by this thread
    const uint32_t lane = threadIdx.x - c * tpr;
    const bool active = c < nrep;
    uint8_t* sp = smem + c * stride_b;
    const uint8_t* jb = EA ? jsm : nullptr;
    const uint8_t* tbl = reinterpret_cast<const uint8_t*>(J.temp_of ? s_tblc[active ? c : 0] : s_tbl);
    const uint32_t r = r0 + c;
    const uint32_t instance = J.inst_base + inst;
    Thr T{J.thr[0], J.thr[1], J.thr[2]};
    if (J.temp_of && active) {
        const uint32_t* th = J.thr_temp + 3ull * J.temp_of[slot0 + c];
        T = Thr{th[0], th[1], th[2]};
    }
    const uint32_t k0 = (uint32_t)J.seed, k1 = (uint32_t)(J.seed >> 32);
    const uint64_t ncopies = (uint64_t)J.n_inst * J.R;
    const bool want_final = J.E || J.M || J.hist;
    const UnitWalk wk = make_walk<DIM>(L, lane, tpr);

    const uint32_t nsw = J.nsweeps;
    for (uint32_t s = 0; s <= nsw; ++s) {
        // s == nsw is a measurement-only pass when nothing was swept
        if (s == nsw && nsw != 0) break;
        const bool sweep = s < nsw;
        const bool measure = (J.Eser != nullptr && sweep) || ((sweep ? s + 1 == nsw : true) && want_final);
        const uint32_t t = J.t0 + s;
        int e = 0, m = 0;
        for (uint32_t colour = 0; colour < 2; ++colour) {
            if (!sweep && colour == 0) continue;
            if (active) {
                const PhiloxFixed pf = philox_fix(t, r, c3_word(kPurposeMetro, colour, instance), k0, k1);
                half_sweep_copy<DIM, EA, SWAR, ROWWISE>(sp, jb, L, N, lane, tpr, wk, colour, pf, T, tbl, sweep,
                                               measure && colour == 1, e, m);
            }
            __syncthreads();
        }
        if (measure) {
            if (active) {
                atomicAdd(&acc_e[c], e);
                atomicAdd(&acc_m[c], m);
            }
            __syncthreads();
            if (threadIdx.x < nrep) {
                const uint32_t cc = threadIdx.x;
                const uint64_t slot = slot0 + cc;
                const int E = acc_e[cc], M = acc_m[cc];
                if (J.Eser && sweep) J.Eser[(uint64_t)s * ncopies + slot] = E;
                if (J.Mser && sweep) J.Mser[(uint64_t)s * ncopies + slot] = M;
                const bool last = sweep ? s + 1 == nsw : true;
                if (last) {
                    if (J.E) J.E[slot] = E;
                    if (J.M) J.M[slot] = M;
                    if (J.hist) {
                        atomicAdd(&J.hist[(uint64_t)inst * J.nbins + (uint32_t)((E - J.e_lo) >> 2)], 1u);
                        atomicMin(&J.emin[inst], E);
                        atomicMax(&J.emax[inst], E);
                        unsigned long long* su = J.sums + (uint64_t)inst * 4;
                        const long long el = E, ml = M;
                        atomicAdd(&su[0], (unsigned long long)el);
                        atomicAdd(&su[1], (unsigned long long)(el * el));
                        atomicAdd(&su[2], (unsigned long long)(ml < 0 ? -ml : ml));
                        atomicAdd(&su[3], (unsigned long long)(ml * ml));
                    }
                }
                acc_e[cc] = 0;
                acc_m[cc] = 0;
            }
            __syncthreads();
        }
    }

    // ---- store ----
    if (nsw > 0 || J.dst != J.src || J.parent) {
        if (SWAR) {
            const uint32_t chunks = N >> 3, W = L >> 3, H = N >> 1;
            for (uint32_t idx = threadIdx.x; idx < nrep * chunks; idx += blockDim.x) {
                const uint32_t cc = idx / chunks, ch = idx - cc * chunks;
                const uint32_t row = ch / W;
                const uint32_t y = DIM == 3 ? row % L : row, z = DIM == 3 ? row / L : 0;
                const uint32_t pe = (y + z) & 1u;
                const uint32_t* pl = reinterpret_cast<const uint32_t*>(smem + cc * stride_b);
                const uint32_t ev = pl[pe * (H >> 2) + ch], od = pl[(pe ^ 1u) * (H >> 2) + ch];
                uint2 v;
                v.x = __byte_perm(ev, od, 0x5140);
                v.y = __byte_perm(ev, od, 0x7362);
                *reinterpret_cast<uint2*>(J.dst + (slot0 + cc) * N + (uint64_t)ch * 8) = v;
            }
        } else {
            const uint32_t nw = N >> 2;
            for (uint32_t idx = threadIdx.x; idx < nrep * nw; idx += blockDim.x) {
                const uint32_t cc = idx / nw, wi = idx - cc * nw;
                reinterpret_cast<uint32_t*>(J.dst + (slot0 + cc) * N)[wi] =
                    reinterpret_cast<const uint32_t*>(smem + cc * stride_b)[wi];
            }
        }
    }
}

size_t resident_smem_bytes(const SweepLaunch& P) {
    size_t mx = 0;
    for (int j = 0; j < P.njobs; ++j) {
        const SweepJob& J = P.jobs[j];
        size_t b = (size_t)J.rpc * ((J.N + 15u) & ~15u);
        if (P.ea) b += (P.swar ? 6ull : 3ull) * J.N;
        if (b > mx) mx = b;
    }
    return mx;
}

template <int DIM, bool EA, bool SWAR, bool ROWWISE>
static cudaError_t launch_res(const SweepLaunch& P, uint32_t n_ctas, uint32_t threads, size_t smem,
                              cudaStream_t s) {
    auto kern = k_sweep_resident<DIM, EA, SWAR, ROWWISE>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<n_ctas, threads, smem, s>>>(P);
    count_launch();
    return cudaGetLastError();
}

template <int DIM, bool EA>
static cudaError_t launch_res_dim(const SweepLaunch& P, uint32_t n_ctas, uint32_t threads, size_t smem,
                                  cudaStream_t s) {
    if (!P.swar) return launch_res<DIM, EA, false, false>(P, n_ctas, threads, smem, s);
    return P.rowwise ? launch_res<DIM, EA, true, true>(P, n_ctas, threads, smem, s)
                     : launch_res<DIM, EA, true, false>(P, n_ctas, threads, smem, s);
}

cudaError_t launch_sweep_resident(const SweepLaunch& P, uint32_t n_ctas, uint32_t threads, size_t smem,
                                  cudaStream_t s) {
    if (P.dim == 2 && !P.ea) return launch_res_dim<2, false>(P, n_ctas, threads, smem, s);
    if (P.dim == 3 && !P.ea) return launch_res_dim<3, false>(P, n_ctas, threads, smem, s);
    if (P.dim == 3 && P.ea) return launch_res_dim<3, true>(P, n_ctas, threads, smem, s);
    return cudaErrorInvalidValue;
}

// ---- tiled sweeps of large 2D lattices: shared-memory tiles with a halo ----
// Each CTA loads a (T + 16) x (T + 16) window (an 8-site halo on every side,
// periodic wrap) of one copy into shared memory as colour planes, runs up to 4
// full sweeps on it, and writes back the T x T interior to the other buffer.
// Half-sweep s updates rows [s + 1, W - s - 1) of the window: the region whose
// neighbours are still exact shrinks by one site per half-sweep, so after 2k
// <= 8 half-sweeps the interior equals the two-phase checkerboard sweeps of the
// whole lattice (Sec. 3.1). Halo sites get updated with stale neighbours and
// are discarded. The 8-site halo keeps every plane word aligned with a whole
// Philox call (4 same-colour sites = 8 lattice columns).
template <uint32_t T>
__global__ void __launch_bounds__(256) k_sweep_tiles(const __grid_constant__ TileLaunch P) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ __align__(16) uint32_t s_tbl[8];
    constexpr uint32_t Wd = T + 16, Wg = Wd >> 3, H = (Wd * Wd) >> 1;
    const uint32_t L = P.L, Lw = L >> 3;
    const uint32_t tiles_x = L / T;
    const uint32_t ty = blockIdx.x / tiles_x, tx = blockIdx.x - ty * tiles_x;
    const uint64_t copy = (uint64_t)P.copy0 + blockIdx.y;
    const uint32_t inst = (uint32_t)(copy / P.R), r = (uint32_t)(copy - (uint64_t)inst * P.R);
    const int8_t* src = P.src + copy * (uint64_t)L * L;
    int8_t* dst = P.dst + copy * (uint64_t)L * L;
    const uint32_t y0 = (ty * T + L - 8) % L;  // global row of window row 0
    const uint32_t xw0 = ((tx * T + L - 8) % L) >> 3;  // global 8-column chunk of window chunk 0
    // load with periodic wrap; chunks never straddle the wrap (L % 8 == 0)
    uint32_t* pl = reinterpret_cast<uint32_t*>(smem);
    for (uint32_t idx = threadIdx.x; idx < Wd * Wg; idx += blockDim.x) {
        const uint32_t rr = idx / Wg, cx = idx - rr * Wg;
        uint32_t gy = y0 + rr, gc = xw0 + cx;
        if (gy >= L) gy -= L;
        if (gc >= Lw) gc -= Lw;
        const uint2 v = *reinterpret_cast<const uint2*>(src + (uint64_t)gy * L + 8ull * gc);
        const uint32_t pe = gy & 1u;  // colour of the even columns of this row
        pl[pe * (H >> 2) + idx] = __byte_perm(v.x, v.y, 0x6420);
        pl[(pe ^ 1u) * (H >> 2) + idx] = __byte_perm(v.x, v.y, 0x7531);
    }
    if (threadIdx.x < 8) {
        const int d = 2 - (int)threadIdx.x;
        s_tbl[threadIdx.x] = d <= 0 ? 0xFFFFFFFFu : (d == 1 ? P.thr[0] : P.thr[1]);
    }
    __syncthreads();
    const uint8_t* tbl = reinterpret_cast<const uint8_t*>(s_tbl);
    const uint32_t k0 = (uint32_t)P.seed, k1 = (uint32_t)(P.seed >> 32);
    const uint32_t instance = P.inst_base + inst;
    int e = 0, m = 0;
    for (uint32_t s = 0; s < 2 * P.nsweeps; ++s) {
        const uint32_t colour = s & 1u, t = P.t0 + (s >> 1);
        const PhiloxFixed pf = philox_fix(t, r, c3_word(kPurposeMetro, colour, instance), k0, k1);
        const uint32_t row_lo = s + 1, rows = Wd - 2 * (s + 1);
        for (uint32_t u = threadIdx.x; u < rows * Wg; u += blockDim.x) {
            const uint32_t rr = u / Wg, g = u - rr * Wg;
            const uint32_t row = row_lo + rr;
            uint32_t gy = y0 + row, gc = xw0 + g;
            if (gy >= L) gy -= L;
            if (gc >= Lw) gc -= Lw;
            const uint32_t q = gy * Lw + gc;
            unit_split<2, false, false>(smem, nullptr, Wd, Wd * Wd, row, row, 0, g, colour, pf, tbl, true, e, m, q);
        }
        __syncthreads();
    }
    // store the T x T interior: window rows [8, 8 + T), chunks [1, 1 + T/8)
    constexpr uint32_t Tc = T >> 3;
    for (uint32_t idx = threadIdx.x; idx < T * Tc; idx += blockDim.x) {
        const uint32_t rr = idx / Tc, cx = idx - rr * Tc;
        const uint32_t wrow = rr + 8, wc = cx + 1;
        const uint32_t gy = ty * T + rr, gx = tx * T + 8 * cx;
        const uint32_t pe = gy & 1u;
        const uint32_t ev = pl[pe * (H >> 2) + wrow * Wg + wc], od = pl[(pe ^ 1u) * (H >> 2) + wrow * Wg + wc];
        uint2 v;
        v.x = __byte_perm(ev, od, 0x5140);
        v.y = __byte_perm(ev, od, 0x7362);
        *reinterpret_cast<uint2*>(dst + (uint64_t)gy * L + gx) = v;
    }
}

size_t tile_smem_bytes(uint32_t T) { return (size_t)(T + 16) * (T + 16); }

cudaError_t launch_sweep_tiles(const TileLaunch& P, uint64_t copies, cudaStream_t s) {
    const size_t smem = tile_smem_bytes(P.T);
    if (P.T != 128 && P.T != 256) return cudaErrorInvalidValue;
    auto kern = P.T == 128 ? k_sweep_tiles<128> : k_sweep_tiles<256>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const uint32_t tiles = (P.L / P.T) * (P.L / P.T);
    for (uint64_t c0 = 0; c0 < copies; c0 += 65535) {
        TileLaunch Q = P;
        Q.copy0 = (uint32_t)c0;
        const uint32_t nc = (uint32_t)((copies - c0) < 65535 ? (copies - c0) : 65535);
        kern<<<dim3(tiles, nc), 256, smem, s>>>(Q);
        count_launch();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// ---- global-memory half-sweep (large lattices) ----
// Grid (unit blocks, copies); one unit per thread.
template <int DIM, bool EA, bool SWAR>
__global__ void __launch_bounds__(256) k_halfsweep_global(int8_t* spins, const uint8_t* jbits, uint32_t L,
                                                          uint32_t N, uint32_t R, uint32_t inst_base,
                                                          uint64_t copy0, uint32_t colour, uint32_t t,
                                                          uint32_t k0, uint32_t k1, Thr T) {
    const uint64_t copy = copy0 + blockIdx.y;
    const uint32_t inst = (uint32_t)(copy / R), r = (uint32_t)(copy - (uint64_t)inst * R);
    uint8_t* sp = reinterpret_cast<uint8_t*>(spins + copy * N);
    const uint8_t* jb = EA ? jbits + (uint64_t)inst * 3 * N : nullptr;
    const uint32_t uu = blockIdx.x * blockDim.x + threadIdx.x;
    const PhiloxFixed pf = philox_fix(t, r, c3_word(kPurposeMetro, colour, inst_base + inst), k0, k1);
    int e = 0, m = 0;
    if (SWAR) {
        const uint32_t G = L >> 3;
        if (uu < (N >> 3)) unit_swar<DIM, EA, false>(sp, jb, L, N, uu / G, uu % G, colour, pf, T, true, e, m);
    } else {
        if (uu < (((N >> 1) + 3) >> 2))
            unit_scalar<DIM, EA, false>(reinterpret_cast<int8_t*>(sp), jb, L, N, uu, colour, pf, T, true, e, m);
    }
}

cudaError_t launch_halfsweep_global(const SweepJob& J, int dim, int colour, uint32_t t, cudaStream_t s) {
    const bool swar = (J.L % 8) == 0;
    const bool ea = J.jbits != nullptr;
    const uint32_t units = swar ? (J.N >> 3) : (((J.N >> 1) + 3) >> 2);
    const uint32_t threads = 256;
    const uint32_t bx = (units + threads - 1) / threads;
    const uint64_t copies = (uint64_t)J.n_inst * J.R;
    const Thr T{J.thr[0], J.thr[1], J.thr[2]};
    const uint32_t k0 = (uint32_t)J.seed, k1 = (uint32_t)(J.seed >> 32);
    int8_t* spins = J.dst;
    for (uint64_t c0 = 0; c0 < copies; c0 += 65535) {
        const uint32_t nc = (uint32_t)((copies - c0) < 65535 ? (copies - c0) : 65535);
        dim3 grid(bx, nc);
#define GBMC_HS(D, E, S) \
    k_halfsweep_global<D, E, S><<<grid, threads, 0, s>>>(spins, J.jbits, J.L, J.N, J.R, J.inst_base, c0, colour, t, k0, k1, T)
        if (dim == 2 && !ea) { if (swar) GBMC_HS(2, false, true); else GBMC_HS(2, false, false); }
        else if (dim == 3 && !ea) { if (swar) GBMC_HS(3, false, true); else GBMC_HS(3, false, false); }
        else if (dim == 3 && ea) { if (swar) GBMC_HS(3, true, true); else GBMC_HS(3, true, false); }
        else return cudaErrorInvalidValue;
        count_launch();
#undef GBMC_HS
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace gbmc
