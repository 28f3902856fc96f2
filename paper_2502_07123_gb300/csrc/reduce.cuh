// Deterministic reduction of per-chunk partial sums, shared by the plan
// finalize kernel and the engine's accumulate kernel so that both produce the
// same bits for the same chunking.
#pragma once
#include <cuda_runtime.h>

#include "item.h"

namespace mlmc {

// Sum partials[0, n) in a fixed order: lane c adds chunks c, c + 32, ... in
// turn, then the 32 lane totals meet in an xor butterfly.  Integer sums are
// exact (Sigma Y^2 in 128 bits); every lane returns the same total.  Called by
// all 32 lanes of a warp.  CG: read through L2 only (partials written by
// other CTAs of the running kernel).
template <bool CG = false>
__device__ inline DevSums warp_sum_partials(const Partial *partials, uint32_t n) {
  const uint32_t lane = threadIdx.x & 31;
  int64_t isum = 0;
  uint64_t lo = 0, hi = 0, ns = 0;
  double ds = 0.0, dq = 0.0;
  for (uint32_t c = lane; c < n; c += 32) {
    const Partial *p = partials + c;
    int64_t pi;
    uint64_t plo, phi, pns;
    double pds, pdq;
    if constexpr (CG) {
      pi = (int64_t)__ldcg((const long long *)&p->isum);
      plo = __ldcg((const unsigned long long *)&p->isum2_lo);
      phi = __ldcg((const unsigned long long *)&p->isum2_hi);
      pds = __ldcg(&p->dsum);
      pdq = __ldcg(&p->dsum2);
      pns = __ldcg((const unsigned long long *)&p->nsat);
    } else {
      pi = p->isum; plo = p->isum2_lo; phi = p->isum2_hi; pds = p->dsum; pdq = p->dsum2; pns = p->nsat;
    }
    isum += pi;
    const uint64_t nlo = lo + plo;
    hi += phi + (uint64_t)(nlo < lo);
    lo = nlo;
    ds += pds;
    dq += pdq;
    ns += pns;
  }
  for (int m = 16; m >= 1; m >>= 1) {
    isum += __shfl_xor_sync(0xffffffffu, (long long)isum, m);
    const uint64_t olo = __shfl_xor_sync(0xffffffffu, (unsigned long long)lo, m);
    const uint64_t ohi = __shfl_xor_sync(0xffffffffu, (unsigned long long)hi, m);
    const uint64_t nlo = lo + olo;
    hi += ohi + (uint64_t)(nlo < lo);
    lo = nlo;
    ds += __shfl_xor_sync(0xffffffffu, ds, m);
    dq += __shfl_xor_sync(0xffffffffu, dq, m);
    ns += __shfl_xor_sync(0xffffffffu, (unsigned long long)ns, m);
  }
  DevSums r;
  r.dsum = ds; r.dsum2 = dq; r.isum = isum; r.isum2_lo = lo; r.isum2_hi = hi; r.nsat = ns;
  return r;
}

// Unsigned 128-bit integer to the nearest double (ties to even).
__device__ inline double u128_to_double_rn(unsigned long long lo, unsigned long long hi) {
  if (hi == 0) return __ull2double_rn(lo);
  const int z = __clzll((long long)hi);
  unsigned long long m = z ? ((hi << z) | (lo >> (64 - z))) : hi;
  const unsigned long long rest = z ? (lo << z) : lo;
  m |= (rest != 0ULL) ? 1ULL : 0ULL;   // sticky bit below the 64 kept bits
  return ldexp(__ull2double_rn(m), 64 - z);
}

}  // namespace mlmc
