"""GB300-native Axilrod-Teller three-body engine (multibody multipole method).

Importing the package is cheap: the CUDA library is loaded on first use of
the API functions (see ``api``)."""
