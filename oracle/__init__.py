"""FP64 CPU oracle for SaLF ray-cast rendering -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never does, and the
two share no code; the only common inputs come from the seeded generators in
``synth``.
"""

from .oracle import (  # noqa: F401
    OracleScene,
    build,
    library_path,
    render,
    render_actors,
    refine,
    subdivide_record,
    face_pairs,
    reg_loss,
    secondary_rays,
    voxel_at,
    backward,
    backward_actors,
    conditioned,
    gen_rays,
    trace,
    trace_eps,
    field,
    sh_basis,
    pose_at,
    num_threads,
)
