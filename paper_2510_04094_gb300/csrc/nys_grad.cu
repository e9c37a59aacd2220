// Adjoint gradient (placeholder translation unit; filled below).
#include "nys_internal.cuh"
