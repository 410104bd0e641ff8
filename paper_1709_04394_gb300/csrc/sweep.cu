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
// Spins are bytes +1 (0x01) / -1 (0xFF). For L % 8 == 0 each thread updates a
// row chunk of 8 bytes at a time (the 4 sites of one colour in it use the 4
// words of one Philox call): the byte-wise "down" bit d = (byte >> 1) & 1 of the
// chunk and of its neighbour chunks is combined with byte-parallel xor/add to
// count, per site, the unsatisfied bonds a (s_i J_ij s_j = -1); then
// dE = 4 (dim - a) and the site flips iff dE <= 0 or u <= T(dE). Other L use a
// per-site path with the same words.
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

template <int DIM, bool EA, bool SWAR>
__device__ __forceinline__ void half_sweep_copy(uint8_t* sp, const uint8_t* jb, uint32_t L, uint32_t N,
                                                uint32_t first_unit, uint32_t stride, uint32_t colour,
                                                const PhiloxFixed& pf, const Thr& T, bool flip,
                                                bool measure, int& e, int& m) {
    if (SWAR) {
        const uint32_t G = L >> 3, units = N >> 3;
        if (measure) {
            for (uint32_t uu = first_unit; uu < units; uu += stride)
                unit_swar<DIM, EA, true>(sp, jb, L, N, uu / G, uu % G, colour, pf, T, flip, e, m);
        } else {
            for (uint32_t uu = first_unit; uu < units; uu += stride)
                unit_swar<DIM, EA, false>(sp, jb, L, N, uu / G, uu % G, colour, pf, T, flip, e, m);
        }
    } else {
        const uint32_t units = ((N >> 1) + 3) >> 2;
        int8_t* s8 = reinterpret_cast<int8_t*>(sp);
        if (measure) {
            for (uint32_t uu = first_unit; uu < units; uu += stride)
                unit_scalar<DIM, EA, true>(s8, jb, L, N, uu, colour, pf, T, flip, e, m);
        } else {
            for (uint32_t uu = first_unit; uu < units; uu += stride)
                unit_scalar<DIM, EA, false>(s8, jb, L, N, uu, colour, pf, T, flip, e, m);
        }
    }
}

__device__ __forceinline__ uint32_t padded(uint32_t n) { return (n + 15u) & ~15u; }

// Grid: one CTA per (job, instance, group of rpc replicas). blockDim.x must be
// a multiple of rpc; blockDim.x / rpc threads serve each replica.
template <int DIM, bool EA, bool SWAR>
__global__ void __launch_bounds__(256) k_sweep_resident(const __grid_constant__ SweepLaunch P) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ int acc_e[64], acc_m[64];
    int jid = 0;
    while (jid + 1 < P.njobs && blockIdx.x >= P.cta_begin[jid + 1]) ++jid;
    const SweepJob& J = P.jobs[jid];
    const uint32_t local = blockIdx.x - P.cta_begin[jid];
    const uint32_t inst = local / J.ctas_per_inst;
    const uint32_t r0 = (local - inst * J.ctas_per_inst) * J.rpc;
    const uint32_t nrep = min(J.rpc, J.R - r0);
    const uint32_t N = J.N, L = J.L, stride_b = padded(N);
    const uint64_t slot0 = (uint64_t)inst * J.R + r0;

    // ---- load: copy c of this CTA from src + parent(c) (gather) ----
    {
        const uint32_t words = stride_b >> 2;  // 4-byte words per copy (N % 4 == 0)
        const uint32_t nw = N >> 2;
        for (uint32_t idx = threadIdx.x; idx < nrep * words; idx += blockDim.x) {
            const uint32_t c = idx / words, wi = idx - c * words;
            if (wi >= nw) continue;
            const uint64_t slot = slot0 + c;
            const uint64_t srcslot = J.parent ? (uint64_t)inst * J.R + J.parent[slot] : slot;
            reinterpret_cast<uint32_t*>(smem + c * stride_b)[wi] =
                reinterpret_cast<const uint32_t*>(J.src + srcslot * N)[wi];
        }
        if (EA) {
            const uint8_t* jsrc = J.jbits + (uint64_t)inst * 3 * N;
            uint8_t* jdst = smem + (uint64_t)J.rpc * stride_b;
            const uint32_t nwj = (3 * N) >> 2;
            for (uint32_t idx = threadIdx.x; idx < nwj; idx += blockDim.x)
                reinterpret_cast<uint32_t*>(jdst)[idx] = reinterpret_cast<const uint32_t*>(jsrc)[idx];
        }
    }
    if (threadIdx.x < 64) {
        acc_e[threadIdx.x] = 0;
        acc_m[threadIdx.x] = 0;
    }
    __syncthreads();

    const uint32_t tpr = blockDim.x / J.rpc;
    const uint32_t c = threadIdx.x / tpr;  // copy served by this thread
    const uint32_t lane = threadIdx.x - c * tpr;
    const bool active = c < nrep;
    uint8_t* sp = smem + c * stride_b;
    const uint8_t* jb = EA ? smem + (uint64_t)J.rpc * stride_b : nullptr;
    const uint32_t r = r0 + c;
    const uint32_t instance = J.inst_base + inst;
    const Thr T{J.thr[0], J.thr[1], J.thr[2]};
    const uint32_t k0 = (uint32_t)J.seed, k1 = (uint32_t)(J.seed >> 32);
    const uint64_t ncopies = (uint64_t)J.n_inst * J.R;
    const bool want_final = J.E || J.M || J.hist;

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
                half_sweep_copy<DIM, EA, SWAR>(sp, jb, L, N, lane, tpr, colour, pf, T, sweep,
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
        const uint32_t words = stride_b >> 2, nw = N >> 2;
        for (uint32_t idx = threadIdx.x; idx < nrep * words; idx += blockDim.x) {
            const uint32_t cc = idx / words, wi = idx - cc * words;
            if (wi >= nw) continue;
            reinterpret_cast<uint32_t*>(J.dst + (slot0 + cc) * N)[wi] =
                reinterpret_cast<const uint32_t*>(smem + cc * stride_b)[wi];
        }
    }
}

size_t resident_smem_bytes(const SweepLaunch& P) {
    size_t mx = 0;
    for (int j = 0; j < P.njobs; ++j) {
        const SweepJob& J = P.jobs[j];
        size_t b = (size_t)J.rpc * ((J.N + 15u) & ~15u);
        if (P.ea) b += 3ull * J.N;
        if (b > mx) mx = b;
    }
    return mx;
}

template <int DIM, bool EA, bool SWAR>
static cudaError_t launch_res(const SweepLaunch& P, uint32_t n_ctas, uint32_t threads, size_t smem,
                              cudaStream_t s) {
    auto kern = k_sweep_resident<DIM, EA, SWAR>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<n_ctas, threads, smem, s>>>(P);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_sweep_resident(const SweepLaunch& P, uint32_t n_ctas, uint32_t threads, size_t smem,
                                  cudaStream_t s) {
    if (P.dim == 2 && !P.ea) {
        return P.swar ? launch_res<2, false, true>(P, n_ctas, threads, smem, s)
                      : launch_res<2, false, false>(P, n_ctas, threads, smem, s);
    }
    if (P.dim == 3 && !P.ea) {
        return P.swar ? launch_res<3, false, true>(P, n_ctas, threads, smem, s)
                      : launch_res<3, false, false>(P, n_ctas, threads, smem, s);
    }
    if (P.dim == 3 && P.ea) {
        return P.swar ? launch_res<3, true, true>(P, n_ctas, threads, smem, s)
                      : launch_res<3, true, false>(P, n_ctas, threads, smem, s);
    }
    return cudaErrorInvalidValue;
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
