// Newton's method for Lemma 2 (placeholder translation unit; filled below).
#include "nys_internal.cuh"
