"""GB300-native GPA stall-blame path: packed PC samples -> stall blame ->
speedup advice (Zhou et al., GPA, Sec. 2.1, 4, 5), as sm_103a CUDA kernels
behind the C ABI of include/gpa.h. This package is the ctypes binding and
the build script; the kernels live in csrc/."""
from .gpa import (Context, GpaError, Program, gpa_advise, gpa_arch_default, gpa_blame, gpa_create, gpa_destroy,  # noqa: F401
                  gpa_copy_counts, gpa_exclusive_scan_noalloc, gpa_set_counts,
                  gpa_get_advice, gpa_get_blame, gpa_get_counts, gpa_get_edges, gpa_get_reaching,
                  gpa_ingest_host_samples, gpa_ingest_samples, gpa_launch_count, gpa_load_program,
                  gpa_reset_counts, gpa_set_launch_stats, gpa_sm_model_of_device, gpa_sync_status,
                  gpa_unload_program, header_functions, library, LAUNCH_DTYPE, OPT_NAMES)
