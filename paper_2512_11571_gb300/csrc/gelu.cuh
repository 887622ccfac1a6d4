// GELU in its erf form and its derivative, FP32, for the surrogate's dense
// layers (the tiled and the tcgen05 GEMM epilogues share them, so both
// paths train the same function).
#pragma once

namespace cem {

// GELU(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2
__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }

// GELU'(z) = Phi(z) + z phi(z)
__device__ __forceinline__ float gelu_grad(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

}  // namespace cem
