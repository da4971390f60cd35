"""GB300-native iterative DVM solver for the Shakhov/BGK model equations
(arXiv 1810.00348).  ``kgs`` is the ctypes binding of the C-ABI library
``libkgs.so``; ``inputs`` builds seeded synthetic problems."""
