// Common prelude of the generated per-level headers (generated by codegen.py).
#pragma once
#include <cuda_runtime.h>
