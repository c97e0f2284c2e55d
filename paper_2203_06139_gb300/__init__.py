"""cg: exact gradients of histogram and event fit objectives on GB300.

The compute path is the CUDA library ``libcg`` (hand-written sm_103a
kernels behind a C ABI); ``paper_2203_06139_gb300.cg`` is its thin Python
binding.  ``synth`` holds the seeded input generators.
"""
