// admm_dev.cuh -- device helpers shared by the ADMM kernels and the batched
// round: the quantizer of Eq. (et21) and the master's z/v update.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/pc2.h"

namespace pc2 {

// Gamma2 / Gamma1 of one value: rint((u - zmin) * scale), IEEE double, no
// contraction; out-of-range (or NaN) values flag PC2_ST_QUANT and clamp.
__device__ __forceinline__ uint64_t quant(double u, double zmin, double scale, double qmax, int* status) {
  const double t = __dmul_rn(__dsub_rn(u, zmin), scale);
  double r = rint(t);
  if (!(r >= 0.0 && r <= qmax)) {  // also catches NaN
    atomicOr(status, PC2_ST_QUANT);
    r = r > qmax ? qmax : 0.0;
  }
  return (uint64_t)r;
}

// Eqs. (ty32), (u78): z = S_kappa(v + x), v = v + x - z.
__device__ __forceinline__ void zv_update(double x, double& z, double& v, double kappa) {
  const double a = __dadd_rn(v, x);
  const double zn = a > kappa ? __dsub_rn(a, kappa) : (a < -kappa ? __dadd_rn(a, kappa) : 0.0);
  v = __dsub_rn(a, zn);
  z = zn;
}

}  // namespace pc2
