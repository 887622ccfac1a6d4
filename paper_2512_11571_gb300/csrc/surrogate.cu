// placeholder translation unit, filled by the surrogate kernels
