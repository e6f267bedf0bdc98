"""CPU reference rasterizer (FP64 values, binary32 decisions).

TEST INFRASTRUCTURE ONLY: used by ``tests/``, the package smoke check and the
CPU-baseline leg of ``bench.py``; the product path never imports it.
"""
from .oracle import Oracle, build, exp_f32, exp2_f32, sh_basis_f32, sh_basis_f64, num_threads, set_num_threads, log_taps, insertion, rig_chain  # noqa: F401
from .frequency import box_downsample, dft_energy, frequency_schedule  # noqa: F401
from . import merging  # noqa: F401
