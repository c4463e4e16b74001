"""FP64 CPU oracle for cylindrical-grid SART.

Test infrastructure only: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` are its only users.  It shares no code with the CUDA path.
"""
from .oracle import (  # noqa: F401
    Setup, build, load, pose_matrix, ray, clip, ray_row, project, backproject, row_sums,
    row_nnz, sart, log_transform, num_threads, set_num_threads,
)
