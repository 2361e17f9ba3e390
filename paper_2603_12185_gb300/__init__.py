"""GB300-native batched ComFree contact step (arxiv 2603.12185).

Importing the package is light: the CUDA library binding lives in ``paper_2603_12185_gb300.comfree``
and the seeded scene generators in ``paper_2603_12185_gb300.scenes``.
"""
__all__ = ["scenes", "comfree"]
