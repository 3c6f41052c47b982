"""GB300-native (sm_103a) batch-incremental CP update after SamBaTen
(Gujral, Pasricha, Papalexakis; arxiv 1709.00668).

The compute path is libsambaten.so (hand-written CUDA kernels behind the C ABI
of include/sambaten.h); `sbt` is its Python binding, `synth` the seeded
planted-tensor generator, `build` the nvcc build.  Importing this package does
not load the library; `sbt.lib()` does, and fails loudly when it is missing.
"""
__all__ = ["build", "sbt", "synth"]
