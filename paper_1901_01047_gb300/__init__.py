"""GB300-native CT-AUX walker (DCA++ hot path).

The compute path is the C-ABI library ``libdcawalker.so`` built from
``csrc/``; ``walker.py`` is its thin ctypes binding.  Importing the package
does not load the library; ``walker.load()`` does, and raises if it is
missing.
"""
