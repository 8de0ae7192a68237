// Generated by paper_2007_08555_gb300/codegen.py for lev_max = 8. Do not edit.
#include "mtp_gen_L8.h"
#define MTP_GEN_NS mtpgen_L8
#define MTP_LEVEL_FN mtp_level_ops_L8
#include "mtp_level_impl.cuh"
