// Metropolis sampling of the batched source-plane chi2 on the device: the
// Bayesian fit of Sec. 2.2 (the likelihood exp(-chi2 / 2) of Eq. 6 explored
// by a Markov chain over the parameters of the varying potentials) run as W
// independent chains, one parameter set each, advanced together.
//
// One step: every chain proposes theta' = theta + sigma * z (z standard
// normal), the batch of proposals goes through the source-plane chi2 kernel,
// and each chain moves to theta' when ln u < -(chi2' - chi2) / (2 T)
// (u uniform in (0, 1), T the temperature; a proposal outside the dPIE
// domain has chi2' = NaN and is refused).
//
// Random numbers: Philox4x64-10 (Salmon, Moraes, Dror and Shaw, "Parallel
// random numbers: as easy as 1, 2, 3", SC 2011), a counter-based generator:
// the words for chain w at step s are Philox(counter = (s, w, j, 0),
// key = (seed, 0)) for j = 0..4, 20 64-bit words; each word x gives the
// uniform ((x >> 11) + 1/2) 2^-53; words 0..15 make 8 Box-Muller pairs (the
// first NP normals are used: 14 parameters, or 16 with the members' scaling
// factors), word 16 the acceptance uniform.
#include "lens_device.cuh"

namespace lens {
namespace {

struct U4 {
  unsigned long long w[4];
};

// Philox4x64 with 10 rounds: per round two 64 x 64 -> 128-bit products mix
// the counter words with the key, which is bumped by the Weyl constants.
__device__ __forceinline__ U4 philox4x64_10(U4 c, unsigned long long k0, unsigned long long k1) {
  constexpr unsigned long long M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  constexpr unsigned long long W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned long long hi0 = __umul64hi(M0, c.w[0]), lo0 = M0 * c.w[0];
    const unsigned long long hi1 = __umul64hi(M1, c.w[2]), lo1 = M1 * c.w[2];
    c = U4{{hi1 ^ c.w[1] ^ k0, lo1, hi0 ^ c.w[3] ^ k1, lo0}};
    k0 += W0;
    k1 += W1;
  }
  return c;
}

__device__ __forceinline__ double unit_open(unsigned long long x) {
  return ((double)(x >> 11) + 0.5) * 0x1.0p-53;
}

// Proposals into prop [W][NP] and the acceptance uniforms into ua [W]: one
// thread per (chain, Philox block j = 0..3), each block's four words giving
// two Box-Muller pairs (parameters 4j .. 4j+3 where < NP); the j = 0 thread
// also draws block 4 for the acceptance uniform.  (One thread per chain left
// most SMs idle: 4096 chains are 32 CTAs of 128.)
// The step's counter word is `step`, or *d_step when d_step is not NULL
// (a counter in device memory that the acceptance kernel advances).
template <int NP>
__global__ void k_mcmc_propose(const double *__restrict__ params, const double *__restrict__ sigma, int W,
                               unsigned long long seed, unsigned long long step,
                               const unsigned long long *__restrict__ d_step, double *__restrict__ prop,
                               double *__restrict__ ua) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int w = t >> 2, j = t & 3;
  if (w >= W) return;
  if (d_step) step = *d_step;
  const U4 r = philox4x64_10(U4{{step, (unsigned long long)w, (unsigned long long)j, 0ull}}, seed, 0ull);
  const double two_pi = 6.283185307179586;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int i = 4 * j + 2 * h;  // parameters i, i + 1
    if (i >= NP) break;
    const double rad = sqrt(-2.0 * log(unit_open(r.w[2 * h]))), ang = two_pi * unit_open(r.w[2 * h + 1]);
    const size_t o = (size_t)w * NP + i;
    prop[o] = params[o] + sigma[i] * (rad * cos(ang));
    prop[o + 1] = params[o + 1] + sigma[i + 1] * (rad * sin(ang));
  }
  if (j == 0) ua[w] = unit_open(philox4x64_10(U4{{step, (unsigned long long)w, 4ull, 0ull}}, seed, 0ull).w[0]);
}

// Metropolis acceptance; accepted[w] (when not NULL) records the decision.
// With a device step counter, one thread advances it: the proposal kernel of
// this step has finished reading it (stream order), the next step reads the
// new value.
__global__ void k_mcmc_accept(double *__restrict__ params, double *__restrict__ chi2,
                              const double *__restrict__ prop, const double *__restrict__ ua,
                              const double *__restrict__ chi2_prop, int W, int np, double temperature,
                              int32_t *__restrict__ accepted, unsigned long long *__restrict__ d_step) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (d_step && w == 0) *d_step += 1ull;
  if (w >= W) return;
  const double cp = chi2_prop[w], c0 = chi2[w];
  bool take = false;
  if (isfinite(cp)) take = !isfinite(c0) || log(ua[w]) < -(cp - c0) / (2.0 * temperature);
  if (take) {
    for (int q = 0; q < np; ++q) params[(size_t)w * np + q] = prop[(size_t)w * np + q];
    chi2[w] = cp;
  }
  if (accepted) accepted[w] = take ? 1 : 0;
}

}  // namespace

int launch_mcmc_step(lens_ctx *ctx, const Model *m, const CSet *c, double *d_params, double *d_chi2, int32_t W,
                     const double *d_sigma, double temperature, unsigned long long seed, unsigned long long step,
                     int32_t variant, int32_t np, double *d_scratch, int32_t *d_accepted, cudaStream_t st,
                     unsigned long long *d_step) {
  double *prop = d_scratch, *ua = d_scratch + (size_t)W * np, *chi2_prop = ua + W;
  const int blocks = (W + 127) / 128, pblocks = (4 * W + 127) / 128;
  if (np == 16)
    k_mcmc_propose<16><<<pblocks, 128, 0, st>>>(d_params, d_sigma, W, seed, step, d_step, prop, ua);
  else
    k_mcmc_propose<14><<<pblocks, 128, 0, st>>>(d_params, d_sigma, W, seed, step, d_step, prop, ua);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(LENS_ECUDA, "proposal launch: %s", cudaGetErrorString(e));
  const int rc = np == 16 ? launch_chi2_source_scaled(ctx, m, c, prop, W, variant, chi2_prop, st)
                          : launch_chi2_source(ctx, m, c, prop, W, variant, chi2_prop, st);
  if (rc) return rc;
  k_mcmc_accept<<<blocks, 128, 0, st>>>(d_params, d_chi2, prop, ua, chi2_prop, W, np, temperature, d_accepted,
                                        d_step);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(LENS_ECUDA, "acceptance launch: %s", cudaGetErrorString(e));
  return LENS_OK;
}

}  // namespace lens
