// Launch-shape table of the autotuner (tune.cpp): host-only, no CUDA types.
#pragma once

namespace mpcg {
namespace tune {

// The tunable launch shapes: streaming-kernel blocks (orthogonalisation,
// update, residual), block-SpMM blocks, window-Gram chunks per window block,
// and the one-point-per-thread Jacobi switch of a grid (1 on, 0 off).
enum { kStream = 0, kSpmm = 1, kGram = 2, kJacobi = 3, kNumTunables = 4 };

// Arithmetic of a keyed shape; kAny for shapes shared by every precision
// (those that size reduction buffers used by the FP64 refinement as well).
enum { kAny = -1, kF32 = 0, kF64 = 1, kDW = 2 };

// The tuned value for the key, or dflt when none is set.
int lookup(int fn, int kind, long long npts, int nb, int C, int dflt);
bool find(int fn, int kind, long long npts, int nb, int C, int* value);
void set(int fn, int kind, long long npts, int nb, int C, int value);
void erase(int fn, int kind, long long npts, int nb, int C);
void clear();
int size();
// JSON cache tagged with the device name and SM count.  save: false on an I/O
// error.  load: entries read (>= 0), -1 no file, -2 malformed, -3 written for
// another device or SM count (nothing is loaded then).
bool save(const char* path, const char* device, int sm_count);
int load(const char* path, const char* device, int sm_count);

}  // namespace tune
}  // namespace mpcg
