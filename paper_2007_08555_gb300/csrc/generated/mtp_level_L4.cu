// Generated by paper_2007_08555_gb300/codegen.py for lev_max = 4. Do not edit.
#include "mtp_gen_L4.h"
#define MTP_GEN_NS mtpgen_L4
#define MTP_LEVEL_FN mtp_level_ops_L4
#include "mtp_level_impl.cuh"
