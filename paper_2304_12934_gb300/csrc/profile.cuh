// Kernel ids of the event profiler (profile.cu) and the launch bracketing
// helpers used by every launcher.
#pragma once
#include <cuda_runtime.h>

enum {
    TCK_FWD_COL = 0, TCK_FWD_ROW, TCK_FWD_DET, TCK_ADJ_DET, TCK_ADJ_ROW, TCK_ADJ_COL,
    TCK_PRIOR, TCK_DOTS, TCK_UPDATE, TCK_REDUCE, TCK_SCALAR, TCK_DOT, TCK_SCALE, TCK_FILL,
    TCK_NRM_COL_FWD, TCK_NRM_ROW, TCK_NRM_COL_ADJ, TCK_PRIOR_NEXT, TCK_FIXUP,
    TCK_COUNT
};

int prof_begin(int id, cudaStream_t s);
void prof_end(int h, cudaStream_t s);

// Brackets one kernel launch statement with profiler events.
#define TC_PROFILED(id, stream, ...)           \
    do {                                       \
        const int _ph = prof_begin((id), (stream)); \
        __VA_ARGS__;                           \
        prof_end(_ph, (stream));               \
    } while (0)
