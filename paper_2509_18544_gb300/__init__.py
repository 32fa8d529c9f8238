"""GB300-native SFFT fit and subtraction (delta-basis matching kernel + polynomial background).

``paper_2509_18544_gb300.sfft`` is the Python binding over the C-ABI library ``libsfft.so``
(hand-written CUDA for sm_103a); ``paper_2509_18544_gb300.synth`` draws seeded synthetic
Roman-like inputs.  Importing the package loads neither; the binding loads the library on
first use and raises if it has not been built.
"""
__all__ = ["sfft", "synth"]
