// Host-side launch accounting: a launch counter and, when enabled, a CUDA
// event pair recorded on the launching stream around every kernel.
#pragma once

#include <cuda_runtime.h>

namespace vpgs {
void prof_begin(const char *name, cudaStream_t s);
void prof_end(cudaStream_t s);
}  // namespace vpgs

// VPGS_LAUNCH("name", stream, kernel<<<grid, block, smem, stream>>>(args...));
#define VPGS_LAUNCH(name, stream, ...)      \
    do {                                    \
        ::vpgs::prof_begin((name), (stream)); \
        __VA_ARGS__;                        \
        ::vpgs::prof_end((stream));         \
    } while (0)
