// sweep.cu -- checkerboard Metropolis sweeps (Sec. 3.1, Eq. (8)) of int8
// lattices with per-site Philox words, for the ferromagnet (Eq. (7), J = 1)
// and the bimodal +-J spin glass (Sec. 6). The per-word site updates and the
// shared-memory layout they work on are in units.cuh.
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
#include "check.cuh"
#include "device.cuh"
#include "internal.h"
#include "units.cuh"

namespace gbmc {
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
            // each thread walks the rows row0, row0 + rstep, ... of its word column;
            // in 2D four rows at a time: all four units are loaded and updated
            // before any word is stored (different rows of the colour plane: none
            // reads what another writes), which frees the scheduler to overlap them
            auto step = [&](uint32_t& y, uint32_t& z) {
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
            };
            uint32_t* own = reinterpret_cast<uint32_t*>(sp + colour * (N >> 1));
            uint32_t y = wk.y0, z = wk.z0, row = wk.row0;
            if constexpr (DIM == 3) {
                // 3D: one unit at a time measured faster (six neighbour words and,
                // for +-J, six bond words per unit already fill the registers)
#pragma unroll 4
                for (; row < rows; row += wk.rstep) {
                    unit_split<DIM, EA, MEASURE>(sp, jbc, L, N, row, y, z, wk.g0, colour, pf, tbl, flip, e, m,
                                                 row * W + wk.g0);
                    step(y, z);
                }
            } else {
#pragma unroll 1
                for (; row + 3 * wk.rstep < rows; row += 4 * wk.rstep) {
                    uint32_t ii[4], vv[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const uint32_t rk = row + k * wk.rstep;
                        unit_split<DIM, EA, MEASURE, false>(sp, jbc, L, N, rk, y, z, wk.g0, colour, pf, tbl, flip, e,
                                                            m, rk * W + wk.g0, &ii[k], &vv[k]);
                        step(y, z);
                    }
                    if (flip) {
#pragma unroll
                        for (int k = 0; k < 4; ++k) own[ii[k]] = vv[k];
                    }
                }
                for (; row < rows; row += wk.rstep) {
                    unit_split<DIM, EA, MEASURE>(sp, jbc, L, N, row, y, z, wk.g0, colour, pf, tbl, flip, e, m,
                                                 row * W + wk.g0);
                    step(y, z);
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

// One work unit = one (job, instance, group of rpc replicas). blockDim.x must
// be a multiple of rpc; blockDim.x / rpc threads serve each replica. Shared
// memory: rpc copies (split colour planes when SWAR, else row-major), then
// the instance's bond planes (EA). Starts and ends without a pending barrier:
// the caller separates consecutive units of one CTA with __syncthreads().
template <int DIM, bool EA, bool SWAR, bool ROWWISE>
__device__ __forceinline__ void resident_unit(const SweepLaunch& P, uint32_t unit) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ int acc_e[64], acc_m[64];
    __shared__ __align__(16) uint32_t s_tbl[8];
    __shared__ __align__(16) uint32_t s_tblc[64][8];  // per-copy tables (parallel tempering)
    int jid = 0;
    while (jid + 1 < P.njobs && unit >= P.cta_begin[jid + 1]) ++jid;
    const SweepJob& J = P.jobs[jid];
    const uint32_t local = unit - P.cta_begin[jid];
    const uint32_t inst = local / J.ctas_per_inst;
    const uint32_t r0 = (local - inst * J.ctas_per_inst) * J.rpc;
    // variable populations: only the first nlive[inst] slots hold replicas
    const uint32_t live = J.nlive ? J.nlive[inst] : J.R;
    if (r0 >= live) return;  // uniform over the CTA, before any barrier
    const uint32_t nrep = min(J.rpc, live - r0);
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
            const uint64_t srcslot =
                J.parent ? (uint64_t)inst * J.R + J.parent[GBMC_IDX(slot, (uint64_t)J.n_inst * J.R)] : slot;
            const uint2 v = *reinterpret_cast<const uint2*>(
                J.src + GBMC_IDX(srcslot * N + (uint64_t)ch * 8, (uint64_t)J.n_inst * J.R * N - 7));
            const uint32_t y = DIM == 3 ? row % L : row, z = DIM == 3 ? row / L : 0;
            const uint32_t pe = (y + z) & 1u;
            uint32_t* pl = reinterpret_cast<uint32_t*>(smem + c * stride_b);
            pl[GBMC_IDX(pe * (H >> 2) + ch, N >> 2)] = __byte_perm(v.x, v.y, 0x6420);
            pl[GBMC_IDX((pe ^ 1u) * (H >> 2) + ch, N >> 2)] = __byte_perm(v.x, v.y, 0x7531);
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
                *reinterpret_cast<uint2*>(
                    J.dst + GBMC_IDX((slot0 + cc) * N + (uint64_t)ch * 8, (uint64_t)J.n_inst * J.R * N - 7)) = v;
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

// Grid launch: CTA b runs unit b. Persistent launch (P.work != null): a grid
// of (SMs x resident CTAs) claims units from a counter in order (the host puts
// the jobs with the largest copies first) until all P.total units are taken;
// the last CTA to finish resets the two counters for the next launch, so
// launches that share them must not overlap. Every unit computes the same
// result either way.
// (Separate instantiations: the claim loop costs the grid form registers.)
template <int DIM, bool EA, bool SWAR, bool ROWWISE, bool PERSISTENT>
__global__ void __launch_bounds__(256) k_sweep_resident(const __grid_constant__ SweepLaunch P) {
    if constexpr (!PERSISTENT) {
        resident_unit<DIM, EA, SWAR, ROWWISE>(P, blockIdx.x);
    } else {
        __shared__ uint32_t s_unit[2];
        for (uint32_t it = 0;; ++it) {
            // alternate slots: a unit without replicas returns with no barrier, so
            // the next claim must not overwrite the slot slower threads still read
            if (threadIdx.x == 0) s_unit[it & 1u] = atomicAdd(P.work, 1u);
            // also orders the previous unit's store loop before the next load
            __syncthreads();
            const uint32_t u = s_unit[it & 1u];
            if (u >= P.total) break;
            resident_unit<DIM, EA, SWAR, ROWWISE>(P, u);
        }
        if (threadIdx.x == 0) {
            __threadfence();
            if (atomicAdd(P.work + 1, 1u) == gridDim.x - 1) {
                atomicExch(P.work, 0u);
                atomicExch(P.work + 1, 0u);
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
    auto kern = P.work ? k_sweep_resident<DIM, EA, SWAR, ROWWISE, true> : k_sweep_resident<DIM, EA, SWAR, ROWWISE, false>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    if (P.work) {
        // persistent: as many CTAs as can be resident at once, at most one per unit
        int dev = 0, sms = 0, per_sm = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, (int)threads, smem);
        if (e != cudaSuccess) return e;
        const uint64_t resident = (uint64_t)(per_sm > 0 ? per_sm : 1) * (uint64_t)sms;
        if (resident < n_ctas) n_ctas = (uint32_t)resident;
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
