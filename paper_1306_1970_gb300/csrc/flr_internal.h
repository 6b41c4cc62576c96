// Library-internal helpers shared between translation units (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>

#include "../../include/flr.h"

// Fewest thread blocks flr_solve can run handle h's problem on: a block's slab
// of the p coefficients must fit its shared-memory vectors (-1 if none does).
int flr_min_grid(flr_t h);

// Global-timer span (ns) of the last solve kernel run on handle h (0, 0 if none).
void flr_kernel_span(flr_t h, unsigned long long* t0, unsigned long long* t1);

// What another translation unit may read of a handle: sizes, the column-major
// X (device, storage dtype, column j at j * ldn), y, X^T y, diag(X^T X), the
// graph (stencil row length q2 = p on a chain; symmetric CSR for edge lists).
struct flr_view {
  int device, sm_count;
  cudaStream_t stream;
  int dtype;
  long long n, p, ldn, m;
  int gkind;
  long long q2;
  const void* Xt;
  const double *y, *c, *d;
  double cnorm;
  const long long* rowptr;
  const int* col;
};
bool flr_get_view(flr_t h, flr_view* v);

// A workspace another translation unit attaches to a handle; `release` frees it
// when the handle is destroyed (called with the handle's device current).
void* flr_aux_get(flr_t h);
void flr_aux_set(flr_t h, void* ws, void (*release)(void*));
