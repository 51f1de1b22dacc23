// lbm_internal.h — helpers shared by the translation units of liblbm_mix.so
// (not part of the C ABI; hidden from the library's exported symbols).
#pragma once

#include "../../include/lbm_mix.h"

#define LBM_HIDDEN __attribute__((visibility("hidden")))

// Records a message for lbm_mix_last_error on this thread; returns code.
LBM_HIDDEN int lbm_internal_error(int code, const char* fmt, ...)
    __attribute__((format(printf, 2, 3)));

// Checks p like lbm_mix_create; *Nx_out receives the number of columns.
LBM_HIDDEN int lbm_internal_validate(const lbm_mix_params* p, int* Nx_out);
