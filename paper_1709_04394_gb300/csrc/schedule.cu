// schedule.cu -- adaptive annealing steps (Sec. 5.4 cites adaptive
// temperature steps without fixing them). Reading: the step dbeta is chosen so
// that the current population's energy histogram h(E) and its reweighting to
// beta + dbeta, P1(E) ~ h(E) exp(-dbeta E), overlap by a target,
//   alpha(dbeta) = sum_E min(h(E)/R, P1(E)),
// by bisection (50 halvings of [0, dmax]); or an MLP proposes dbeta from the
// population's energy moments and is accepted when its realised overlap lies
// in a band, the bisection being the fallback. One CTA per lattice.
#include <cuda_bf16.h>

#include "device.cuh"
#include "internal.h"

namespace gbmc {

namespace {

__device__ __forceinline__ float bfr(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// Sum over the block; every thread receives the result. sh: 33 doubles.
__device__ double block_sum_d(double v, double* sh) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    if (warp == 0) {
        double s = lane < nw ? sh[lane] : 0.0;
        s = warp_sum(s);
        if (lane == 0) sh[32] = s;
    }
    __syncthreads();
    const double r = sh[32];
    __syncthreads();
    return r;
}

__device__ double overlap_eval(const uint32_t* h, uint32_t bmin, uint32_t bmax, double R, double d, double* sh) {
    double w = 0.0;
    for (uint32_t b = bmin + threadIdx.x; b <= bmax; b += blockDim.x) {
        const uint32_t hb = h[b];
        if (hb) w += (double)hb * exp(-d * 4.0 * (double)(b - bmin));
    }
    const double W = block_sum_d(w, sh);
    double a = 0.0;
    for (uint32_t b = bmin + threadIdx.x; b <= bmax; b += blockDim.x) {
        const uint32_t hb = h[b];
        if (hb) {
            const double p0 = (double)hb / R;
            const double p1 = (double)hb * exp(-d * 4.0 * (double)(b - bmin)) / W;
            a += p0 < p1 ? p0 : p1;
        }
    }
    return block_sum_d(a, sh);
}

}  // namespace

__global__ void __launch_bounds__(256) k_schedule(const __grid_constant__ SchedLaunch S) {
    __shared__ double sh[33];
    __shared__ float xin[kMlpIn], h1[kMlpHidden], h2[kMlpHidden];
    __shared__ double ys;
    const SchedJob& J = S.jobs[blockIdx.x];
    const int32_t emin = *J.emin, emax = *J.emax;
    const uint32_t bmin = (uint32_t)(emin - J.e_lo) >> 2, bmax = (uint32_t)(emax - J.e_lo) >> 2;
    const double R = (double)J.R;
    // moments of E - Emin
    double s1 = 0.0;
    for (uint32_t b = bmin + threadIdx.x; b <= bmax; b += blockDim.x)
        s1 += (double)J.hist[b] * 4.0 * (double)(b - bmin);
    const double m1 = block_sum_d(s1, sh) / R;
    double s2 = 0.0, s3 = 0.0;
    for (uint32_t b = bmin + threadIdx.x; b <= bmax; b += blockDim.x) {
        const double hb = (double)J.hist[b];
        const double dx = 4.0 * (double)(b - bmin) - m1;
        s2 += hb * dx * dx;
        s3 += hb * dx * dx * dx;
    }
    const double var = block_sum_d(s2, sh) / R;
    const double m3 = block_sum_d(s3, sh) / R;
    double skew = var > 0.0 ? m3 / (var * sqrt(var)) : 0.0;
    skew = skew < -10.0 ? -10.0 : (skew > 10.0 ? 10.0 : skew);
    double f[kMlpIn];
    f[0] = ((double)emin + m1) / (double)J.N;
    f[1] = log(var / (double)J.N + 1e-6);
    f[2] = skew;
    f[3] = J.beta;
    f[4] = log((double)J.L);
    f[5] = log(R);

    int kind = 1, evals = 0;
    double dbeta = 0.0, alpha = 1.0, proposal = 0.0, alpha_p = 0.0;
    if (S.mode == 2 && S.mlp) {
        const float* p = S.mlp;
        if (threadIdx.x < kMlpIn) xin[threadIdx.x] = (float)f[threadIdx.x];
        __syncthreads();
        if (threadIdx.x < kMlpHidden) {
            const int j = threadIdx.x;
            float a = bfr(p[kOffB1 + j]);
            for (int i = 0; i < kMlpIn; ++i) a += bfr(p[kOffW1 + j * kMlpIn + i]) * xin[i];
            h1[j] = tanhf(a);
        }
        __syncthreads();
        if (threadIdx.x < kMlpHidden) {
            const int j = threadIdx.x;
            float a = bfr(p[kOffB2 + j]);
            for (int k = 0; k < kMlpHidden; ++k) a += bfr(p[kOffW2 + j * kMlpHidden + k]) * h1[k];
            h2[j] = tanhf(a);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            float y = bfr(p[kOffB3]);
            for (int j = 0; j < kMlpHidden; ++j) y += bfr(p[kOffW3 + j]) * h2[j];
            ys = (double)y;
        }
        __syncthreads();
        // output y = log(dbeta sigma_E)
        const double sigma = sqrt(var > 1e-12 ? var : 1e-12);
        proposal = exp(ys) / sigma;
        if (proposal > J.dmax) proposal = J.dmax;
        alpha_p = overlap_eval(J.hist, bmin, bmax, R, proposal, sh);
        ++evals;
        if (S.lo <= alpha_p && alpha_p <= S.hi) {
            kind = 2;
            dbeta = proposal;
            alpha = alpha_p;
        }
    }
    int clamped = 0;
    if (kind == 1) {
        const double amax = overlap_eval(J.hist, bmin, bmax, R, J.dmax, sh);
        ++evals;
        if (amax >= S.target) {
            dbeta = J.dmax;
            alpha = amax;
        } else {
            double lo = 0.0, hi = J.dmax, alo = 1.0;
            for (int it = 0; it < 50; ++it) {
                const double mid = 0.5 * (lo + hi);
                const double a = overlap_eval(J.hist, bmin, bmax, R, mid, sh);
                ++evals;
                if (a >= S.target) {
                    lo = mid;
                    alo = a;
                } else {
                    hi = mid;
                }
            }
            dbeta = lo;
            alpha = alo;
        }
    }
    clamped = dbeta == J.dmax;
    if (threadIdx.x == 0) {
        SchedOut& o = S.out[blockIdx.x];
        o.dbeta = dbeta;
        o.alpha = alpha;
        o.proposal = proposal;
        o.alpha_proposal = alpha_p;
        o.var = var;
        for (int i = 0; i < kMlpIn; ++i) o.feat[i] = (float)f[i];
        o.kind = kind;
        o.clamped = clamped;
        o.evals = evals;
        o.emin = emin;
        o.emax = emax;
        o.pad = 0;
    }
}

cudaError_t launch_schedule(const SchedLaunch& S, cudaStream_t s) {
    k_schedule<<<S.njobs, 256, 0, s>>>(S);
    count_launch();
    return cudaGetLastError();
}

}  // namespace gbmc
