"""GB300 (sm_103a) library for replica-averaged Brownian dynamics
(Kania, Nguyen, Oztekin & Webb, arXiv 2206.05851).

- ``bdra``: Python binding of the C ABI declared in include/bdra.h.
- ``inputs``: seeded synthetic inputs (initial coils, workload tables).
- ``build``: compiles csrc/ into libbdra.so for sm_103a.
"""
