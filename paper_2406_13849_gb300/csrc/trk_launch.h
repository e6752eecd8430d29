// trk_launch.h - launchers shared between the kernel translation units
// (not part of the ABI).
#pragma once
#include <cuda_runtime.h>

#include "trk.h"
#include "trk_device.cuh"
#include "trk_internal.h"

namespace trk {

// Rays per block of the transmission kernels (128 threads, 8 rays each); the
// backward pass keeps one row of partial sums per block in its work buffer.
constexpr long long TRK_RAYS_PER_BLOCK = 1024;

// Event kernel: CTAs to launch for `slots` particle slots per CTA (fills the
// GPU at the kernel's occupancy), and the work bytes that needs.
int event_grid(int slots);
size_t event_work_bytes(int slots, int grid);
// TRK_OK if the geometry fits the event kernels' slot record (the CSG or the
// array tracker), else TRK_E_UNSUPPORTED (with the message set, naming
// `where`, unless where is NULL).
trk_status event_fits(trk_geom_t g, bool csg, const char* where);

trk_status launch_event(trk_geom_t g, const ParticlesView& P, long long n, const dev::RunP& rp, bool csg, bool f32,
                        int flags,
                        unsigned long long* tally, unsigned long long* cnt, unsigned long long* rec, void* work,
                        size_t work_bytes, int slots, int grid, int max_rounds, int sort_interval, cudaStream_t s);

}  // namespace trk
