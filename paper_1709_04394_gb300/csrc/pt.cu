// pt.cu -- replica exchange of parallel tempering (Sec. 5.1, Eq. (10)).
// Temperatures k = 0..T-1 (ascending beta) of every instance hold one
// configuration each; round n proposes the pairs (k, k+1) with k = n mod 2,
// n mod 2 + 2, ... . With a = configuration at k, b at k+1, the swap is
// accepted with probability min(1, exp((beta_k - beta_{k+1})(E_a - E_b))):
// always when E_b >= E_a, else iff the pair's Philox word (purpose 4: q = k>>2,
// word k&3, t = n, r = 0) is <= the host-computed threshold of the energy gap
// E_a - E_b = 4m. Swaps exchange temperature labels (rep_of / temp_of), not
// configurations, as the paper recommends for shared memory.
#include "device.cuh"
#include "internal.h"

namespace gbmc {

__global__ void k_pt_exchange(const __grid_constant__ PtExchange X) {
    const uint32_t inst = blockIdx.x;
    uint32_t* rep = X.rep_of + (uint64_t)inst * X.T;
    uint32_t* tmp = X.temp_of + (uint64_t)inst * X.T;
    const int32_t* E = X.E + (uint64_t)inst * X.T;
    for (uint32_t k = 2 * threadIdx.x + (X.round & 1u); k + 1 < X.T; k += 2 * blockDim.x) {
        const uint32_t a = rep[k], b = rep[k + 1];
        const int32_t Ea = E[a], Eb = E[b];
        bool accept = Eb >= Ea;
        if (!accept) {
            const uint32_t m = (uint32_t)(Ea - Eb) >> 2;
            const long long thr = X.tab[(uint64_t)k * (X.M + 1) + (m <= X.M ? m : X.M)];
            const uint4 w = philox4x32_10(make_uint4(k >> 2, X.round, 0u, (4u << 28) | (X.inst_base + inst)),
                                          (uint32_t)X.seed, (uint32_t)(X.seed >> 32));
            const uint32_t u = word_of(w, k & 3u);
            accept = (long long)u <= thr;
        }
        if (accept) {
            rep[k] = b;
            rep[k + 1] = a;
            tmp[b] = k;
            tmp[a] = k + 1;
            X.accepted[(uint64_t)inst * (X.T - 1) + k] += 1u;
        }
    }
}

cudaError_t launch_pt_exchange(const PtExchange& X, cudaStream_t s) {
    if (X.T < 2) return cudaSuccess;
    k_pt_exchange<<<X.n_inst, 128, 0, s>>>(X);
    count_launch();
    return cudaGetLastError();
}

}  // namespace gbmc
