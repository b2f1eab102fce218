// admm_dev.cuh -- device helpers shared by the ADMM kernels and the batched
// round: the quantizer of Eq. (et21) and the master's z/v update.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/pc2.h"

namespace pc2 {

// Gamma2 / Gamma1 of one value: rint((u - zmin) * scale), IEEE double, no
// contraction; out-of-range (or NaN) values flag PC2_ST_QUANT and clamp
// (above the range to qmax, below it and NaN to 0; a value that rounds to
// -0 is 0 without a flag).  scale is a power of two, so after the one
// rounded subtraction d = u - zmin the product d * scale and its rounding to
// an integer (half to even) are exact operations on d's bits, done here with
// integer instructions: B300 runs FP64 at a small fraction of its integer rate.
__device__ __forceinline__ uint64_t quant(double u, double zmin, double scale, double qmax, int* status) {
  const double d = __dsub_rn(u, zmin);
  const long long b = __double_as_longlong(d);
  const int ex = (int)((b >> 52) & 0x7ff);
  const uint64_t frac = (uint64_t)b & ((1ull << 52) - 1u);
  const int ks = (int)((__double_as_longlong(scale) >> 52) & 0x7ff) - 1023;  // scale = 2^ks
  const uint64_t qm = (uint64_t)qmax;
  bool bad;
  uint64_t r;
  if (ex == 0x7ff) {  // infinities and NaN
    bad = true;
    r = (frac == 0u && b >= 0) ? qm : 0u;
  } else {
    const uint64_t m = ex ? (frac | (1ull << 52)) : frac;
    const int s = (ex ? ex : 1) - 1075 + ks;  // |d| * scale = m * 2^s exactly
    uint64_t R = 0;
    bool over = false;
    if (m != 0u) {
      if (s >= 0) {
        over = (64 - __clzll((long long)m)) + s > 64;
        if (!over) R = m << s;
      } else if (-s < 64) {
        const int sh = -s;
        const uint64_t q = m >> sh, rem = m & ((1ull << sh) - 1u), half = 1ull << (sh - 1);
        R = q + ((rem > half || (rem == half && (q & 1u))) ? 1u : 0u);
      }  // else |d| * scale < 2^53 / 2^64 rounds to 0
    }
    if (b < 0) {  // d < 0: rint gives -0 (accepted) or a negative integer
      bad = over || R != 0u;
      r = 0u;
    } else {
      bad = over || R > qm;
      r = bad ? qm : R;
    }
  }
  if (bad) atomicOr(status, PC2_ST_QUANT);
  return r;
}

// Eqs. (ty32), (u78): z = S_kappa(v + x), v = v + x - z.  The two comparisons
// with +-kappa (kappa >= 0) read a's bit pattern (the magnitude ordering of
// non-NaN doubles is the integer ordering of their bits); z = a - sign(a) kappa
// is the same IEEE operation as a - kappa or a + kappa.
__device__ __forceinline__ void zv_update(double x, double& z, double& v, double kappa) {
  const double a = __dadd_rn(v, x);
  const long long ab = __double_as_longlong(a), kb = __double_as_longlong(kappa);
  const long long mag = ab & 0x7fffffffffffffffLL;
  const bool outside = mag > kb && mag <= 0x7ff0000000000000LL;  // |a| > kappa, a not NaN
  const double ksg = __longlong_as_double(kb | (ab & (long long)0x8000000000000000ULL));
  const double zn = outside ? __dsub_rn(a, ksg) : 0.0;
  v = __dsub_rn(a, zn);
  z = zn;
}

}  // namespace pc2
