"""CPU oracle of the DS-PHD/MIB filter -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package.  It shares no code with the CUDA path.
"""
from .oracle import OracleFilter, philox4x32_10, box_muller, ln_f32, sincos2pi_f32, exp_f32, cell_update, radar_likelihood  # noqa: F401
