"""FP64 CPU oracle for RBRP (arXiv 2309.16002) -- test infrastructure only.

Only tests/, __graft_entry__.smoke() and the CPU legs of bench.py may import
this package.  It shares no code with the CUDA library and imports nothing from
it; the product path fails loudly when its CUDA extension is missing instead of
falling back here.

Modules:
  philox  Philox4x64-10 (published definition) and the sampler's uniforms
  rbrp    Alg. 1 (SRP), Alg. 2 (RBRP/BRP/RBGP), Alg. 3 and the W alternatives

Every function is pinned by tests under tests/ marked "not gpu"; none is
"parity unpinned".
"""
from . import philox, rbrp  # noqa: F401
