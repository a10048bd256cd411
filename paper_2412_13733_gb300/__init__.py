"""hpG on one GB300: a C-ABI CUDA library (libhpg) and its thin Python binding.

``paper_2412_13733_gb300.hpg`` loads ``libhpg.so`` (built in-tree by
``paper_2412_13733_gb300.build``); ``workloads`` holds the seeded problem data.
"""
