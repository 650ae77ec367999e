"""GB300-native 1D-3V PIC-MCC thermionic He diode (arXiv 2605.07083)."""
