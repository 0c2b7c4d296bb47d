"""VoGE renderer hot path on GB300 (sm_103a): C-ABI library ``libvoge.so`` and its Python binding.

``scenes`` (seeded synthetic inputs) imports without the CUDA library; the
renderer entry points live in ``paper_2205_15401_gb300.voge`` and load
``libvoge.so`` on first use, failing loudly if it has not been built.
"""
