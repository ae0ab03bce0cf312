"""Array BP-XOR coded matrix multiplication on one GB300 (sm_103a).

``bpx`` is the Python binding of the C-ABI library ``libbpx.so`` (built by
``build.build()``); ``workloads`` holds the seeded synthetic inputs.
"""
from . import bpx  # noqa: F401
