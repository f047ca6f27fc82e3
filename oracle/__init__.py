"""FP64 CPU oracle -- test infrastructure only.

Imported only by ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference leg of ``bench.py``.  The product path (``paper_1704_00512_gb300``)
never imports, links or runs anything here, and this package never imports the
product path.
"""
from . import ref  # noqa: F401
