// okz_batch_internal.h -- device-side slot table of the batched kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "okz_internal.h"

namespace okz {

// One slot: a lattice (height-parity plane) in the batch arena.
struct SlotDesc {
  uint64_t seed;
  uint64_t P, Q;
  int32_t k;
  int32_t L;
  uint32_t t;       // completed sweeps
  uint32_t active;
  uint64_t offset_words;  // lattice position in the arena (32-bit words)
  long long H0;           // h(0,0)
  unsigned long long sum[8];  // exact S_1..S_4 of (h - H0) as (lo, hi) pairs
};

struct WorkItem {
  int32_t slot;
  int32_t sweeps;
};

// count items follow the header; capacity is the batch's slot count.
struct WorkTable {
  int32_t count;
  int32_t pad;
  WorkItem item[1];
};

inline size_t work_table_bytes(int capacity) {
  return sizeof(WorkTable) + (size_t)(capacity > 1 ? capacity - 1 : 0) * sizeof(WorkItem);
}

constexpr int64_t kBatchMaxL = 8192;  // largest lattice one CTA takes on

cudaError_t launch_batch_sweeps(uint32_t *arena, SlotDesc *slots, const WorkTable *work,
                                unsigned int *head, int grid, int threads, size_t smem_bytes,
                                cudaStream_t st);
cudaError_t launch_batch_moments(const uint32_t *arena, SlotDesc *slots, const WorkTable *work,
                                 int nitems, int64_t max_L, cudaStream_t st);
int batch_occupancy(int threads, size_t smem_bytes);

}  // namespace okz
