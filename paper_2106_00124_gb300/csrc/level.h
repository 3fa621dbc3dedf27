// level.h -- the level-batched schedule of a batch of excluded sums
// (exsum_level.cu), as used by the batch planner (exsum_batch.cu).  Internal
// to the library.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "../../include/exsum.h"

namespace exsum {

// Tuning of a level set (0 = the default of each field).
struct LevelTune {
    int lc = 0;           // rows per strided-pass chunk: 0 = sized per tensor, else 16 .. 128
    int interleave = 1;   // level 1: each tensor's row-total pieces next to the strided chunks over the same rows
    int tiles_per_vb = 2; // bulk final pass: tiles per virtual block (the row-to-block assignment)
    int tall = 0;         // k_rowx final pass: tallest tiles (1) or tiles sized for one tensor alone (0)
    int persist = 0;      // persistent grids pulling slots from a counter (1), or one block per slot (0)
};

struct LevelSet;

// Streaming multiprocessors of the current device.
int level_sms();

// Whether the descriptor can join a level set.
bool level_accepts(const exsum_desc &d, int sms);

// Plans descs[idx[0..n-1]] (all accepted) as one level set: allocates its
// workspace and device work lists.  Streams and events for the parallel
// branches are created here, outside any capture.
int level_create(const exsum_desc *descs, const int *idx, int n, const LevelTune &tune, LevelSet **out);

// Enqueues the level set on `s` (capturable): at most thirteen kernels (and,
// for persistent grids, one memset of the work-list counters), in up to
// three parallel branches.
int level_enqueue(LevelSet *ls, cudaStream_t s);

size_t level_workspace_bytes(const LevelSet *ls);
int level_kernels(const LevelSet *ls);
void level_destroy(LevelSet *ls);

}  // namespace exsum
