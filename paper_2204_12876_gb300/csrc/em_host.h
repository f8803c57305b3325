// em_host.h -- host-side internals shared by the translation units of libem.so
// (the map object itself stays private to em_api.cu).
#pragma once

#include <cuda_runtime.h>

#include "em.h"
#include "em_internal.cuh"

namespace em {

int map_device(const em_map* m);
uint32_t map_flags(const em_map* m);
int32_t map_cells(const em_map* m);
const em_params& map_params(const em_map* m);

// Start one update of map m: advances its update index and returns its
// device descriptor (pt_begin / pt_count are left to the caller).
MapDev map_begin_update(em_map* m, int64_t points);
void map_end_update(em_map* m, cudaStream_t s, int64_t points);
void map_undo_update(em_map* m, int64_t points);

// Copy layers, ring offsets, shift and update index of src into dst (same size).
int map_copy_state(em_map* dst, const em_map* src, cudaStream_t s);

// Write the layers in mask (em_get_layers layout) to dst, a pointer the device
// can write (device memory or mapped page-locked host memory), on stream s.
int map_read_layers(em_map* m, uint32_t mask, float* dst, cudaStream_t s);
// The same for n maps, kMaxReadJobs per launch.
int maps_read_layers(em_map* const* maps, const uint32_t* masks, float* const* dst, int n, cudaStream_t s);

// Record a CUDA error for em_last_cuda_error() and map it to a status code.
int map_record_error(const char* what, cudaError_t e);

}  // namespace em
