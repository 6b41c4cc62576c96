// Library-internal helpers shared between translation units (not part of the C ABI).
#pragma once
#include "../../include/flr.h"

// Global-timer span (ns) of the last solve kernel run on handle h (0, 0 if none).
void flr_kernel_span(flr_t h, unsigned long long* t0, unsigned long long* t1);
