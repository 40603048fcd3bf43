"""CPU FP64 oracle for the NASGabor appearance path (arXiv 2606.09794).

TEST INFRASTRUCTURE ONLY. Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package. It is a
plain restatement of the paper's definitions in float64 numpy and shares no
code with the CUDA library (``paper_2606_09794_gb300``), which never imports it.

Modules:
  nasgabor  -- NASGabor lobe, appearance model forward/backward (Sec. 4.2, 5.1, Supp. C/E/F)
  sh        -- real spherical harmonics forward/backward (Sec. 3.2)
  adam      -- Adam update, fused BF16 step and the teacher/student fitting step
  frustum   -- pinhole visibility of primitive centres
  schedule  -- the camera k-NN learning-rate heuristic and the cosine LR schedule
  raster    -- front-to-back alpha compositing of the primitives (the colours' consumer)

Parity pins: every function here is checked in ``tests/test_oracle_*.py``
against closed forms, special cases that reduce to textbook or library
routines, invariances and central finite differences.
"""
from . import adam, frustum, nasgabor, raster, schedule, sh  # noqa: F401
