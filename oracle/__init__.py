"""Plain, slow, float64 CPU oracle of the formal solution and its acceleration structure.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA path (``paper_2511_08498_gb300``) and never imports it; both read
their inputs from the seeded generators in ``synth``.

Modules:
  lc     -- long-characteristics formal solution (C core, ``lc_dense.c``)
  mips   -- sparsity map, Morton block layout, VLM MIP chain and expansion
  lc3, mips3 -- the same in 3D (C core ``lc3_dense.c``; 8^3 blocks, 2x2x2 groups)
  rc     -- radiance-cascade formal solution (interval core ``rc_dense.c``)
  lines  -- MIP-0 emissivity/opacity of the static continuum + line model

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(3D: ``tests/test_oracle3_pins.py``; cascades: ``tests/test_oracle_rc_pins.py``)
(closed forms, exact rational geometry, brute force, printed values of the
paper) except where its docstring says "parity unpinned".
"""

from . import lc, lc3, mips, mips3, lines, rc  # noqa: F401
