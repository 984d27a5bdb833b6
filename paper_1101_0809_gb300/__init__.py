"""GB300-native charge-conserving PIC step (alternating-order gather, relativistic
push, virtual-path deposit) after Sokolov, arXiv:1101.0809.

The compute path is the CUDA library ``libpic.so`` built from ``csrc/`` and
reached through the C ABI declared in ``include/pic.h``; ``pic`` is its Python
binding (argument marshalling only).
"""
__all__ = ["pic", "workloads"]
