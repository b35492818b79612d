// Launch choices measured on the GPU by paper_1208_4869_gb300/autotune.py
// (rerun it with --write to regenerate this file; measured on NVIDIA GB300).
// Each entry: for solves of precision `dtype` (CCG_C64 / CCG_C128) by
// `method` on a dense operator of order n <= nmax (the first matching entry
// wins), whether the solve runs as one persistent launch (1) or as the
// kernel-per-step loop (0), and the persistent launch's blocks per SM (0:
// the occupancy limit).
#pragma once

namespace ccg {

struct TuneEntry {
  int dtype, method;
  long long nmax;
  int persistent, pk_blocks;
};

static const TuneEntry kTune[] = {
    {0, 0, 128, 1, 1},   // complex64 bicgstab n <= 128
    {0, 0, 4611686018427387904, 0, 0},   // complex64 bicgstab n <= any
    {0, 1, 4611686018427387904, 0, 0},   // complex64 cgnr n <= any
    {0, 2, 256, 0, 0},   // complex64 qmr n <= 256
    {0, 2, 512, 1, 1},   // complex64 qmr n <= 512
    {0, 2, 4611686018427387904, 0, 0},   // complex64 qmr n <= any
    {0, 3, 128, 1, 1},   // complex64 cocg n <= 128
    {0, 3, 256, 0, 0},   // complex64 cocg n <= 256
    {0, 3, 512, 1, 1},   // complex64 cocg n <= 512
    {0, 3, 4611686018427387904, 0, 0},   // complex64 cocg n <= any
    {1, 0, 4611686018427387904, 0, 0},   // complex128 bicgstab n <= any
    {1, 1, 4611686018427387904, 0, 0},   // complex128 cgnr n <= any
    {1, 2, 4611686018427387904, 0, 0},   // complex128 qmr n <= any
    {1, 3, 4611686018427387904, 0, 0},   // complex128 cocg n <= any
};

}  // namespace ccg
