"""GB300-native asynchronous randomized Kaczmarz (AsyRK, arXiv:1401.4780).

Importing the package loads nothing compiled.  ``paper_1401_4780_gb300.asyrk``
is the ctypes binding of the C-ABI library ``libasyrk.so`` (built in-tree by
``__graft_entry__.build()``); ``paper_1401_4780_gb300.synth`` generates seeded
synthetic systems.
"""
__all__ = ["asyrk", "synth"]
