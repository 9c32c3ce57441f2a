"""GB300-native (sm_103a) linearization of the voxelized-GICP matching cost factor
of arXiv 2202.00242 (Sec. III-A).

    from paper_2202_00242_gb300 import api     # torch-facing calls over the C ABI
    from paper_2202_00242_gb300 import synth   # seeded synthetic workloads

The compute path is the CUDA library ``libvgicp_gb300.so`` (C ABI in
``include/vgicp.h``), built by ``paper_2202_00242_gb300.build``.
"""
__all__ = ["api", "synth", "build"]
