// lattice.cu -- initial configurations (Sec. 3.1 step 1), bimodal couplings
// (Sec. 6) and the observables E (Eq. (7)) and M of int8 lattices.
#include "device.cuh"
#include "internal.h"

namespace gbmc {

// One thread per group of 4 consecutive sites of one copy: the INIT word of
// q = site>>2 gives all four spins (s = +1 iff the word's top bit is 0).
__global__ void k_init_spins(uint32_t* spins4, uint32_t N4, uint32_t L, uint32_t R, uint64_t ncopies,
                             uint32_t inst_base, uint32_t k0, uint32_t k1, int random_start) {
    const uint64_t total = ncopies * (uint64_t)N4;
    for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < total;
         g += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t copy = g / N4;
        const uint32_t q = (uint32_t)(g - copy * N4);
        uint32_t packed = 0x01010101u;
        if (random_start) {
            const uint32_t inst = (uint32_t)(copy / R), r = (uint32_t)(copy - (uint64_t)inst * R);
            const uint4 w = philox4x32_10(make_uint4(q, 0u, r, c3_word(kPurposeInit, 0u, inst_base + inst)), k0, k1);
            packed = ((w.x >> 31) ? 0xFFu : 0x01u) | (((w.y >> 31) ? 0xFFu : 0x01u) << 8) |
                     (((w.z >> 31) ? 0xFFu : 0x01u) << 16) | (((w.w >> 31) ? 0xFFu : 0x01u) << 24);
        }
        spins4[g] = packed;
    }
}

cudaError_t launch_init_spins(int8_t* spins, int dim, uint32_t L, uint32_t n_inst, uint32_t R,
                              uint32_t inst_base, uint64_t seed, int random_start, cudaStream_t s) {
    uint64_t N = L;
    for (int d = 1; d < dim; ++d) N *= L;
    const uint64_t ncopies = (uint64_t)n_inst * R;
    const uint64_t total = ncopies * (N / 4);
    const uint32_t threads = 256;
    const uint64_t blocks = (total + threads - 1) / threads;
    const uint32_t grid = (uint32_t)(blocks < 152ull * 64 ? blocks : 152ull * 64);
    k_init_spins<<<grid, threads, 0, s>>>(reinterpret_cast<uint32_t*>(spins), (uint32_t)(N / 4), L, R,
                                          ncopies, inst_base, (uint32_t)seed, (uint32_t)(seed >> 32),
                                          random_start);
    count_launch();
    return cudaGetLastError();
}

// Couplings: bond b = 3*site + mu, word b&3 of q = b>>2 (t = r = 0). Stored as
// three byte planes per instance, [inst][mu][site], byte 1 where J = -1.
__global__ void k_couplings(uint8_t* jbits, uint32_t N, uint32_t n_inst, uint32_t inst_base,
                            uint32_t k0, uint32_t k1) {
    const uint64_t total = (uint64_t)n_inst * N;
    for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < total;
         g += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t inst = (uint32_t)(g / N), site = (uint32_t)(g - (uint64_t)inst * N);
        const uint32_t c3 = c3_word(kPurposeCoupling, 0u, inst_base + inst);
#pragma unroll
        for (uint32_t mu = 0; mu < 3; ++mu) {
            const uint64_t b = 3ull * site + mu;
            const uint4 w = philox4x32_10(make_uint4((uint32_t)(b >> 2), 0u, 0u, c3), k0, k1);
            const uint32_t u = word_of(w, (uint32_t)(b & 3));
            jbits[((uint64_t)inst * 3 + mu) * N + site] = (uint8_t)(u >> 31);
        }
    }
}

cudaError_t launch_couplings(uint8_t* jbits, uint32_t L, uint32_t n_inst, uint32_t inst_base,
                             uint64_t seed, cudaStream_t s) {
    const uint32_t N = L * L * L;
    const uint64_t total = (uint64_t)n_inst * N;
    const uint32_t threads = 256;
    uint64_t blocks = (total + threads - 1) / threads;
    if (blocks > 152ull * 32) blocks = 152ull * 32;
    k_couplings<<<(uint32_t)blocks, threads, 0, s>>>(jbits, N, n_inst, inst_base, (uint32_t)seed,
                                                      (uint32_t)(seed >> 32));
    count_launch();
    return cudaGetLastError();
}

// jsplit[((inst*2 + c)*6 + d)*(N/2) + row*(L/2) + j] = 4 if the bond in
// direction d of the colour-c site (row, j) has J = -1. Directions: the x
// neighbour with the same plane index j, the other x neighbour, y-1, y+1,
// z-1, z+1. The site is x = 2j + o with o = (y+z+c)&1: for o = 0 the same-j
// neighbour is x+1 and the other x-1; for o = 1 the reverse.
__global__ void k_split_bonds(const uint8_t* jbits, uint8_t* jsplit, uint32_t L, uint32_t n_inst) {
    const uint32_t N = L * L * L, H = N / 2;
    const uint64_t total = (uint64_t)n_inst * N;  // (inst, c, row, j)
    for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < total;
         g += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t inst = (uint32_t)(g / N);
        const uint32_t rem = (uint32_t)(g - (uint64_t)inst * N);
        const uint32_t c = rem / H, k = rem - c * H;
        const uint32_t row = k / (L / 2), j = k - row * (L / 2);
        const uint32_t y = row % L, z = row / L;
        const uint32_t o = (y + z + c) & 1u;
        const uint32_t x = 2 * j + o;
        const uint8_t* Jx = jbits + (uint64_t)inst * 3 * N;
        const uint8_t* Jy = Jx + N;
        const uint8_t* Jz = Jx + 2 * N;
        const uint32_t site = row * L + x;
        const uint32_t xm = row * L + (x == 0 ? L - 1 : x - 1);
        const uint32_t ym = (z * L + (y == 0 ? L - 1 : y - 1)) * L + x;
        const uint32_t zm = ((z == 0 ? L - 1 : z - 1) * L + y) * L + x;
        const uint8_t fwd_x = Jx[site], bwd_x = Jx[xm];
        uint8_t b[6];
        b[0] = o ? bwd_x : fwd_x;
        b[1] = o ? fwd_x : bwd_x;
        b[2] = Jy[ym];
        b[3] = Jy[site];
        b[4] = Jz[zm];
        b[5] = Jz[site];
        uint8_t* dst = jsplit + ((uint64_t)inst * 2 + c) * 6 * H + k;
#pragma unroll
        for (int d = 0; d < 6; ++d) dst[(uint64_t)d * H] = b[d] ? 4 : 0;
    }
}

cudaError_t launch_split_bonds(const uint8_t* jbits, uint8_t* jsplit, uint32_t L, uint32_t n_inst,
                               cudaStream_t s) {
    k_split_bonds<<<152 * 8, 256, 0, s>>>(jbits, jsplit, L, n_inst);
    count_launch();
    return cudaGetLastError();
}

__global__ void k_jbits_to_int8(const uint8_t* jbits, int8_t* out, uint32_t N, uint32_t n_inst) {
    const uint64_t total = (uint64_t)n_inst * N * 3;
    for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < total;
         g += (uint64_t)gridDim.x * blockDim.x) {
        // out layout [inst][site][mu]
        const uint64_t inst = g / (3ull * N);
        const uint64_t rem = g - inst * 3ull * N;
        const uint64_t site = rem / 3, mu = rem % 3;
        out[g] = jbits[(inst * 3 + mu) * N + site] ? -1 : 1;
    }
}

cudaError_t launch_jbits_to_int8(const uint8_t* jbits, int8_t* out, uint32_t N, uint32_t n_inst,
                                 cudaStream_t s) {
    k_jbits_to_int8<<<152 * 8, 256, 0, s>>>(jbits, out, N, n_inst);
    count_launch();
    return cudaGetLastError();
}

// E = -sum_i sum_mu J_{i,mu} s_i s_{i+mu} (forward bonds), M = sum_i s_i.
// Grid (blocks per copy, copies); each block covers a contiguous site range.
__global__ void k_observables(const int8_t* spins, const uint8_t* jbits, int dim, uint32_t L,
                              uint32_t N, uint32_t R, uint32_t sites_per_block, uint64_t copy0,
                              int32_t* E, int32_t* M) {
    const uint64_t copy = copy0 + blockIdx.y;
    const uint32_t inst = (uint32_t)(copy / R);
    const int8_t* s = spins + copy * N;
    const uint8_t* jb = jbits ? jbits + (uint64_t)inst * 3 * N : nullptr;
    const uint32_t begin = blockIdx.x * sites_per_block;
    const uint32_t end = min(N, begin + sites_per_block);
    int e = 0, m = 0;
    for (uint32_t i = begin + threadIdx.x; i < end; i += blockDim.x) {
        const uint32_t x = i % L, y = (i / L) % L, z = dim == 3 ? i / (L * L) : 0;
        const int si = s[i];
        const uint32_t xr = (x + 1 == L) ? 0 : x + 1, yr = (y + 1 == L) ? 0 : y + 1;
        const uint32_t row = dim == 3 ? (z * L) : 0;
        const int sx = s[(row + y) * L + xr];
        const int sy = s[(row + yr) * L + x];
        int jx = 1, jy = 1, jz = 1;
        if (jb) {
            jx = jb[i] ? -1 : 1;
            jy = jb[N + i] ? -1 : 1;
            jz = jb[2 * N + i] ? -1 : 1;
        }
        int bond = jx * sx + jy * sy;
        if (dim == 3) {
            const uint32_t zr = (z + 1 == L) ? 0 : z + 1;
            bond += jz * s[(zr * L + y) * L + x];
        }
        e -= si * bond;
        m += si;
    }
    e = warp_sum(e);
    m = warp_sum(m);
    __shared__ int se[32], sm[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        se[warp] = e;
        sm[warp] = m;
    }
    __syncthreads();
    if (warp == 0) {
        e = lane < (int)(blockDim.x >> 5) ? se[lane] : 0;
        m = lane < (int)(blockDim.x >> 5) ? sm[lane] : 0;
        e = warp_sum(e);
        m = warp_sum(m);
        if (lane == 0) {
            if (gridDim.x == 1) {
                if (E) E[copy] = e;
                if (M) M[copy] = m;
            } else {
                if (E) atomicAdd(&E[copy], e);
                if (M) atomicAdd(&M[copy], m);
            }
        }
    }
}

cudaError_t launch_observables(const int8_t* spins, const uint8_t* jbits, int dim, uint32_t L,
                               uint32_t n_inst, uint32_t R, int32_t* E, int32_t* M, cudaStream_t s) {
    uint32_t N = L * L * (dim == 3 ? L : 1);
    const uint32_t spb = 65536;
    const uint32_t bx = (N + spb - 1) / spb;
    const uint64_t copies = (uint64_t)n_inst * R;
    if (bx > 1) {
        if (E) { cudaError_t e = cudaMemsetAsync(E, 0, sizeof(int32_t) * copies, s); if (e) return e; }
        if (M) { cudaError_t e = cudaMemsetAsync(M, 0, sizeof(int32_t) * copies, s); if (e) return e; }
    }
    // blockIdx.y is limited to 65535: larger copy counts take several launches
    for (uint64_t c0 = 0; c0 < copies; c0 += 65535) {
        const uint32_t nc = (uint32_t)((copies - c0) < 65535 ? (copies - c0) : 65535);
        dim3 grid(bx, nc);
        k_observables<<<grid, 256, 0, s>>>(spins, jbits, dim, L, N, R, spb, c0, E, M);
        count_launch();
        cudaError_t e = cudaGetLastError();
        if (e) return e;
    }
    return cudaSuccess;
}

}  // namespace gbmc
