// placeholder translation unit, filled by the batched scheduler
