"""MLCC3 triples path on GB300 (sm_103a): C-ABI CUDA library + thin binding.

Importing the package does not load the CUDA library; ``binding.load()`` (or
``binding.Context``) does, and fails loudly when it has not been built.
"""
__all__ = ["binding", "build", "synth"]
